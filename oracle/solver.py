"""The FDLB time step for the simplified Enskog equation in cylindrical and spherical
geometry, written out plainly in FP64 (paper Secs. II-III).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State: weighted populations f[c, i, j, k] (Sec. III.A population formula) on N radial cells,
i over the 2 Q_R half-range radial momenta (positive half first), j and k over the full-range
momenta of the two homogeneous axes: (phi, z) for the cylinder, (theta, phi) for the sphere.

The right-hand side L(f) = -advection - force + collision (A1 reading of the collision sign):

* advection (Sec. II.B/C, conservative form): finite volume in R,
  adv_c = (A_{c+1/2} F_{c+1/2} - A_{c-1/2} F_{c-1/2}) / V_c, F = p_R * WENO5-JS reconstruction
  of f/w upwinded by sign(p_R), epsilon = 1e-6;
* force (Sec. II.B/C curvature terms, Sec. III.B matrices): cylinder
  kappa [p_phi^2 K^h f - p_R K2_phi f]; sphere kappa/2 [(p_th^2 + p_ph^2) K^h f - p_r (K2_th f + K2_ph f)],
  kappa = (A_+ - A_-)/V (about 1/R for the cylinder, 2/r for the sphere);
* collision (Eqs. j0, j1, Shakhov f^S): -(f - f^S)/tau + J1[f^MB] with the covariant strain
  (A2 reading), chi from the Fischer-Methfessel density (RET-FM) or the local density (SET);
* diffuse walls at the faces of the computational domain (Sec. IV): incoming directions carry
  n_w times the wall Maxwellian on the half-range axis, n_w from zero net mass flux; two ghost
  cells per side (incoming: wall Maxwellian, outgoing: cubic extrapolation in the cell index).

Time stepping: the three-stage TVD (SSP) Runge-Kutta scheme of Shu and Osher (Sec. III).

Reduced cylinder (``reduced=True``; the p_z axis integrated out at the level of the model
equation, Sec. III.A's remark on the trivial axes of Couette flow): the pair phi = int f dp_z,
chi = int p_z^2 f dp_z on the (p_R, p_phi) quadrature, stored as f[c, i, j, 0] and f[c, i, j, 1].
With f even in p_z (u_z = q_z = 0, no strain involving z), advection and the curvature force act
on each member as on f (neither involves p_z); the moments need p_z only through
int p_z^2 f = sum chi; the collision of each member is the p_z-integral of the full one, which
replaces the p_z^2 carried by xi^2 with T (phi) or 3T (chi, from int p_z^4 g = 3 T^2) and weights
chi's equilibrium by T.  The diffuse walls emit the wall Maxwellian pair (1, T_w) and balance the
mass flux of phi alone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import equilibrium as eq
from . import geometry as geo
from . import kmatrix as km
from . import model
from . import quadrature as quad

RET_FM = 0
SET_LOCAL = 1
WENO_EPS = 1e-6
RK3_COEFFS = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))  # f_out = a f^n + b (f + dt L(f))


@dataclass
class Problem:
    geometry: int
    grid: geo.Grid
    pR: np.ndarray
    wR: np.ndarray
    alphaR: np.ndarray
    betaR: np.ndarray
    p2: np.ndarray
    w2: np.ndarray
    p3: np.ndarray
    w3: np.ndarray
    NR: int
    N2: int
    N3: int
    KR: np.ndarray
    K2: np.ndarray
    K3: np.ndarray
    sigma: float
    eta0: float
    n0: float
    chi_model: int
    W: np.ndarray
    dt: float
    T_wall: tuple = (1.0, 1.0)     # (inner, outer)
    u_wall: tuple = (0.0, 0.0)     # tangential speed on axis 2 (cylinder only)
    extra: dict = field(default_factory=dict)
    reduced: bool = False          # cylinder with p_z integrated out: f[..., 0] = phi, f[..., 1] = chi

    @property
    def shape(self):
        return (self.grid.N, len(self.pR), len(self.p2), len(self.p3))

    @property
    def w(self):
        return self.wR[:, None, None] * self.w2[None, :, None] * self.w3[None, None, :]


def default_order(Q):
    """Expansion order N_a = min(Q_a - 1, 7) (A6 reading; Sec. III.C requires N_a < Q_a)."""
    return min(Q - 1, 7)


def make_problem(geometry, R_in, R_out, n_cells, Q_R, Q_2, Q_3, eta0, Kn=None, sigma=None,
                 beta=0.0, N_R=None, N_2=None, N_3=None, chi_model=RET_FM,
                 T_wall=(1.0, 1.0), u_wall=(0.0, 0.0), dt=None, cfl=0.4, n_gl=32, reduced=False):
    """reduced: the cylinder with p_z integrated out (Q_3 is then ignored; the third index holds
    the pair phi, chi)."""
    L = R_out - R_in
    if sigma is None:
        _, sigma, n0 = model.physical_parameters(Kn, eta0, L)
    else:
        n0 = 6.0 * eta0 / (math.pi * sigma ** 3)
    grid = geo.make_grid(geometry, R_in, R_out, sigma, n_cells, beta)
    xR, lamR, aR, bR = quad.half_range_rule(Q_R)
    pR = np.concatenate([xR, -xR])
    wR = np.concatenate([lamR, lamR])
    p2, w2 = quad.full_range_rule(Q_2)
    NR = default_order(Q_R) if N_R is None else N_R
    N2 = default_order(Q_2) if N_2 is None else N_2
    KR = km.k1_half(pR, wR, aR, bR)
    K2 = km.k2_full(p2, w2)
    if reduced:
        assert geometry == geo.CYL
        # the pair (phi, chi): no p_z nodes; unit weights, so WENO works on phi / (w_R w_2) and chi / (w_R w_2)
        p3, w3, N3, K3 = np.zeros(2), np.ones(2), 0, np.zeros((2, 2))
    else:
        p3, w3 = quad.full_range_rule(Q_3)
        N3 = default_order(Q_3) if N_3 is None else N_3
        K3 = km.k2_full(p3, w3)
    W = geo.fm_weights(grid, sigma, n_gl) if chi_model == RET_FM else np.zeros((0, 0))
    if dt is None:
        dr_min = float(np.min(np.diff(grid.R_f)))
        Tmax = max(T_wall)
        chi0 = float(model.chi_set(eta0))
        tau_min = float(model.relaxation_time(n0, Tmax, chi0, sigma))
        dt = min(cfl * dr_min / (float(np.max(np.abs(pR))) * math.sqrt(Tmax)), 0.5 * tau_min)
    return Problem(geometry, grid, pR, wR, aR, bR, p2, w2, p3, w3, NR, N2, N3, KR, K2, K3,
                   sigma, eta0, n0, chi_model, W, float(dt), tuple(T_wall), tuple(u_wall), reduced=reduced)


# ----------------------------------------------------------------------------- moments
def momentum_axes(P: Problem):
    return (P.pR[:, None, None], P.p2[None, :, None], P.p3[None, None, :])


def raw_sums(f, P: Problem):
    """The 13 quadrature sums per cell (Eq. mom_quad): S0 = sum f, S1_a = sum f p_a,
    S2_ab = sum f p_a p_b (a <= b: 00, 11, 22, 01, 02, 12), S3_a = sum f p^2 p_a."""
    if P.reduced:
        return _raw_sums_reduced(f, P)
    p = momentum_axes(P)
    psq = p[0] ** 2 + p[1] ** 2 + p[2] ** 2
    ax = (1, 2, 3)
    out = [f.sum(ax)]
    out += [(f * p[a]).sum(ax) for a in range(3)]
    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
        out.append((f * (p[a] * p[b])).sum(ax))
    out += [(f * (psq * p[a])).sum(ax) for a in range(3)]
    return np.stack(out, axis=-1)  # (N, 13)


def _raw_sums_reduced(f, P: Problem):
    """The same 13 sums from the reduced pair: p_z enters only through sum_z p_z^2 f = sum chi
    (S2_zz, and S3_a's p^2 p_a); with f even in p_z its odd moments (S1_z, S2_Rz, S2_phiz, S3_z)
    vanish."""
    phi, chi = f[..., 0], f[..., 1]
    pR, p2 = P.pR[None, :, None], P.p2[None, None, :]
    ax = (1, 2)
    zero = np.zeros(f.shape[0])
    psq = pR ** 2 + p2 ** 2
    out = [phi.sum(ax), (phi * pR).sum(ax), (phi * p2).sum(ax), zero,
           (phi * pR ** 2).sum(ax), (phi * p2 ** 2).sum(ax), chi.sum(ax), (phi * pR * p2).sum(ax), zero, zero,
           (phi * psq * pR).sum(ax) + (chi * pR).sum(ax), (phi * psq * p2).sum(ax) + (chi * p2).sum(ax), zero]
    return np.stack(out, axis=-1)


def macroscopic(S):
    """n, u, T, q and the second-moment matrix from the raw sums (Eq. macro_def):
    u = S1/n, T = (tr S2 - n u^2)/(3n), q_a = (S3_a - 2 u_b S2_ab - u_a tr S2 + 2 n u^2 u_a)/2."""
    n = S[..., 0]
    u = S[..., 1:4] / n[..., None]
    M2 = np.empty(S.shape[:-1] + (3, 3))
    for idx, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        M2[..., a, b] = M2[..., b, a] = S[..., 4 + idx]
    tr = M2[..., 0, 0] + M2[..., 1, 1] + M2[..., 2, 2]
    u2 = (u * u).sum(-1)
    T = (tr - n * u2) / (3.0 * n)
    q = 0.5 * (S[..., 10:13] - 2.0 * np.einsum("...ab,...b->...a", M2, u) - u * tr[..., None]
               + 2.0 * (n * u2)[..., None] * u)
    return n, u, T, q, M2


def moments(f, P: Problem):
    """Dictionary of per-cell n, u (3), T, q (3) and the shear stress P_{R,2} = M2_01 - n u_0 u_1."""
    n, u, T, q, M2 = macroscopic(raw_sums(f, P))
    return {"n": n, "u": u, "T": T, "q": q, "P01": M2[..., 0, 1] - n * u[..., 0] * u[..., 1]}


# ----------------------------------------------------------------------------- closure
def d_dR(phi, grid: geo.Grid):
    """Fourth-order central difference in the mapped coordinate s, divided by dR/ds;
    one-sided five-point fourth-order stencils at the two cells next to each wall (A9)."""
    N = len(phi)
    h = grid.ds
    d = np.empty(N)
    d[2:N - 2] = (phi[0:N - 4] - 8.0 * phi[1:N - 3] + 8.0 * phi[3:N - 1] - phi[4:N]) / (12.0 * h)
    d[0] = (-25.0 * phi[0] + 48.0 * phi[1] - 36.0 * phi[2] + 16.0 * phi[3] - 3.0 * phi[4]) / (12.0 * h)
    d[1] = (-3.0 * phi[0] - 10.0 * phi[1] + 18.0 * phi[2] - 6.0 * phi[3] + phi[4]) / (12.0 * h)
    d[N - 2] = (3.0 * phi[N - 1] + 10.0 * phi[N - 2] - 18.0 * phi[N - 3] + 6.0 * phi[N - 4] - phi[N - 5]) / (12.0 * h)
    d[N - 1] = (25.0 * phi[N - 1] - 48.0 * phi[N - 2] + 36.0 * phi[N - 3] - 16.0 * phi[N - 4] + 3.0 * phi[N - 5]) / (12.0 * h)
    return d / grid.dRds_c


def closure(f, P: Problem):
    """Per-cell quantities of the collision operator (Sec. II):
    n, u, T, q; nbar (Eq. fm) and chi (Eq. chi / chi_ret); b rho (local n); tau (Eq. tau);
    Pr (Eq. prandtl); the gradients of J1 (Eq. j1) by `d_dR`; the covariant strain S_ab and
    div u (A2 reading); the per-axis equilibrium vectors g_R, g_2, g_3 (Sec. III.C)."""
    G = P.grid
    n, u, T, q, _ = macroscopic(raw_sums(f, P))
    if P.chi_model == RET_FM:
        nbar = P.W @ n
        chi = model.chi_set(model.eta_of_n(nbar, P.sigma))
    else:
        nbar = n.copy()
        chi = model.chi_set(model.eta_of_n(n, P.sigma))
    br = model.b_rho(n, P.sigma)
    Pr = model.prandtl(n, chi, P.sigma)
    tau = model.relaxation_time(n, T, chi, P.sigma)
    X = d_dR(np.log(n * n * chi * T), G)
    Y = d_dR(np.log(T), G)
    du = np.stack([d_dR(u[:, a], G) for a in range(3)], axis=-1)
    R = G.R_c
    S = np.zeros((G.N, 3, 3))
    S[:, 0, 0] = du[:, 0]
    if P.geometry == geo.CYL:
        S[:, 1, 1] = u[:, 0] / R
        S[:, 0, 1] = S[:, 1, 0] = 0.5 * (du[:, 1] - u[:, 1] / R)
        S[:, 0, 2] = S[:, 2, 0] = 0.5 * du[:, 2]
        div = du[:, 0] + u[:, 0] / R
    else:
        S[:, 1, 1] = S[:, 2, 2] = u[:, 0] / R
        S[:, 0, 1] = S[:, 1, 0] = 0.5 * (du[:, 1] - u[:, 1] / R)
        S[:, 0, 2] = S[:, 2, 0] = 0.5 * (du[:, 2] - u[:, 2] / R)
        div = du[:, 0] + 2.0 * u[:, 0] / R
    gR = eq.g_half(P.pR, P.wR, P.alphaR, P.betaR, P.NR, u[:, 0], T)
    g2 = eq.g_full(P.p2, P.w2, P.N2, u[:, 1], T)
    g3 = eq.g_full(P.p3, P.w3, P.N3, u[:, 2], T)
    return dict(n=n, u=u, T=T, q=q, nbar=nbar, chi=chi, br=br, Pr=Pr, tau=tau, X=X, Y=Y,
                S=S, div=div, gR=gR, g2=g2, g3=g3)


def collision(f, P: Problem, cl):
    """C = -(f - f^S)/tau + J1[f^MB] evaluated at the node momenta (A5 reading):
    f^MB = n g_R g_2 g_3;  f^S = f^MB [1 + (1 - Pr)/(n T^2) (xi^2/(5T) - 1) xi.q]  (Eq. fmb, Shakhov);
    J1 = -b rho chi f^MB { xi_R [X + 3/5 (zeta^2 - 5/2) Y] + 2/5 [2 zeta_a zeta_b S_ab + (zeta^2 - 5/2) div u] }
    with zeta = xi / sqrt(2T)  (Eq. j1)."""
    p = momentum_axes(P)
    e = lambda a: a[:, None, None, None]
    n, T, u, q = cl["n"], cl["T"], cl["u"], cl["q"]
    xi = [p[a][None] - e(u[:, a]) for a in range(3)]
    xi2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    xiq = xi[0] * e(q[:, 0]) + xi[1] * e(q[:, 1]) + xi[2] * e(q[:, 2])
    fMB = e(n) * cl["gR"][:, :, None, None] * cl["g2"][:, None, :, None] * cl["g3"][:, None, None, :]
    fS = fMB * (1.0 + e((1.0 - cl["Pr"]) / (n * T * T)) * (xi2 / (5.0 * e(T)) - 1.0) * xiq)
    zeta2 = xi2 / (2.0 * e(T))
    strain = np.zeros_like(xi2)
    for a in range(3):
        for b in range(3):
            strain = strain + xi[a] * xi[b] * e(cl["S"][:, a, b])
    strain = 2.0 * strain / (2.0 * e(T))  # 2 zeta_a zeta_b S_ab
    J1 = -e(cl["br"] * cl["chi"]) * fMB * (
        xi[0] * (e(cl["X"]) + 0.6 * (zeta2 - 2.5) * e(cl["Y"]))
        + 0.4 * (strain + (zeta2 - 2.5) * e(cl["div"])))
    return -(f - fS) / e(cl["tau"]) + J1


def collision_reduced(f, P: Problem, cl):
    """The collision of the reduced pair: the p_z-integral of the full operator against 1 (phi)
    and p_z^2 (chi) for the Gaussian p_z factor of f^MB (u_z = 0): int g_z = 1, int p_z^2 g_z = T,
    int p_z^4 g_z = 3 T^2.  Every p_z-dependence of f^S / f^MB and J1 / f^MB is through p_z^2 in
    xi^2 (q_z = 0, and the strain has no z component in the cylinder), so member k is the
    full expression with p_z^2 replaced by e_k = T (phi) or 3T (chi), times m_k = 1 or T."""
    e = lambda a: a[:, None, None]
    n, T, u, q = cl["n"], cl["T"], cl["u"], cl["q"]
    xi0 = P.pR[None, :, None] - e(u[:, 0])
    xi1 = P.p2[None, None, :] - e(u[:, 1])
    xiq = xi0 * e(q[:, 0]) + xi1 * e(q[:, 1])
    fMB = e(n) * cl["gR"][:, :, None] * cl["g2"][:, None, :]
    S = cl["S"]
    strain_perp = (xi0 ** 2 * e(S[:, 0, 0]) + xi1 ** 2 * e(S[:, 1, 1]) + 2.0 * xi0 * xi1 * e(S[:, 0, 1])) / e(T)
    out = np.empty_like(f)
    for k, (ez, mk) in enumerate(((T, np.ones_like(T)), (3.0 * T, T))):
        xi2 = xi0 ** 2 + xi1 ** 2 + e(ez)
        fS = e(mk) * fMB * (1.0 + e((1.0 - cl["Pr"]) / (n * T * T)) * (xi2 / (5.0 * e(T)) - 1.0) * xiq)
        zeta2 = xi2 / (2.0 * e(T))
        J1 = -e(cl["br"] * cl["chi"] * mk) * fMB * (
            xi0 * (e(cl["X"]) + 0.6 * (zeta2 - 2.5) * e(cl["Y"])) + 0.4 * (strain_perp + (zeta2 - 2.5) * e(cl["div"])))
        out[..., k] = -(f[..., k] - fS) / e(cl["tau"]) + J1
    return out


# ----------------------------------------------------------------------------- advection
def weno5(vm2, vm1, v0, vp1, vp2):
    """WENO5-JS (Jiang & Shu 1996) value at the right face of the centre cell v0, upwind
    from the left; the mirror case is obtained by reversing the arguments."""
    b0 = 13.0 / 12.0 * (vm2 - 2.0 * vm1 + v0) ** 2 + 0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) ** 2
    b1 = 13.0 / 12.0 * (vm1 - 2.0 * v0 + vp1) ** 2 + 0.25 * (vm1 - vp1) ** 2
    b2 = 13.0 / 12.0 * (v0 - 2.0 * vp1 + vp2) ** 2 + 0.25 * (3.0 * v0 - 4.0 * vp1 + vp2) ** 2
    q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0
    q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0
    q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0
    a0 = 0.1 / (WENO_EPS + b0) ** 2
    a1 = 0.6 / (WENO_EPS + b1) ** 2
    a2 = 0.3 / (WENO_EPS + b2) ** 2
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def wall_maxwellians(P: Problem):
    """Weighted wall Maxwellians (inner, outer): g^h_R(0, T_w) g^H_2(u_w, T_w) g^H_3(0, T_w)."""
    out = []
    for side in (0, 1):
        Tw, uw = P.T_wall[side], P.u_wall[side]
        gR = eq.g_half(P.pR, P.wR, P.alphaR, P.betaR, P.NR, 0.0, Tw)
        g2 = eq.g_full(P.p2, P.w2, P.N2, uw, Tw)
        # reduced pair: (int g_z, int p_z^2 g_z) = (1, T_w)
        g3 = np.array([1.0, Tw]) if P.reduced else eq.g_full(P.p3, P.w3, P.N3, 0.0, Tw)
        out.append(gR[:, None, None] * g2[None, :, None] * g3[None, None, :])
    return out


def advection(f, P: Problem, return_walls=False):
    """Conservative radial advection with diffuse walls (module docstring)."""
    G = P.grid
    N = G.N
    w = P.w
    v = f / w[None]
    pos = P.pR > 0
    neg = ~pos
    ext = np.empty((N + 4,) + f.shape[1:])
    ext[2:N + 2] = v
    # outgoing ghosts: cubic extrapolation from the four cells next to the wall
    ext[1] = 4 * v[0] - 6 * v[1] + 4 * v[2] - v[3]
    ext[0] = 10 * v[0] - 20 * v[1] + 15 * v[2] - 4 * v[3]
    ext[N + 2] = 4 * v[N - 1] - 6 * v[N - 2] + 4 * v[N - 3] - v[N - 4]
    ext[N + 3] = 10 * v[N - 1] - 20 * v[N - 2] + 15 * v[N - 3] - 4 * v[N - 4]
    X = lambda c: ext[c + 2]  # cell index c in [-2, N+1]
    gw = wall_maxwellians(P)
    pRb = P.pR[:, None, None]
    # the mass flux: of every population, or of phi alone for the reduced pair
    mass = (lambda a: a[..., :1]) if P.reduced else (lambda a: a)
    # left wall: outgoing = p_R < 0, reconstructed from the right at face 0
    vhat_L = weno5(X(2), X(1), X(0), X(-1), X(-2))
    out_L = mass((np.abs(pRb) * w * vhat_L)[neg]).sum()
    in_L = mass((pRb * gw[0])[pos]).sum()
    nw_L = out_L / in_L
    # right wall: outgoing = p_R > 0, reconstructed from the left at face N
    vhat_R = weno5(X(N - 3), X(N - 2), X(N - 1), X(N), X(N + 1))
    out_R = mass((pRb * w * vhat_R)[pos]).sum()
    in_R = mass((np.abs(pRb) * gw[1])[neg]).sum()
    nw_R = out_R / in_R
    # incoming ghosts: the wall Maxwellian
    for c in (-1, -2):
        ext[c + 2][pos] = (nw_L * gw[0] / w)[pos]
    for c in (N, N + 1):
        ext[c + 2][neg] = (nw_R * gw[1] / w)[neg]
    # face values (weighted populations) at faces 0..N
    face = np.empty((N + 1,) + f.shape[1:])
    k = np.arange(1, N)
    left = weno5(ext[k - 3 + 2], ext[k - 2 + 2], ext[k - 1 + 2], ext[k + 2], ext[k + 1 + 2])
    right = weno5(ext[k + 2 + 2], ext[k + 1 + 2], ext[k + 2], ext[k - 1 + 2], ext[k - 2 + 2])
    face[1:N] = np.where(pos[None, :, None, None], left, right) * w[None]
    face[0] = np.where(pos[:, None, None], nw_L * gw[0], w * vhat_L)
    face[N] = np.where(pos[:, None, None], w * vhat_R, nw_R * gw[1])
    F = G.A_f[:, None, None, None] * pRb[None] * face
    adv = (F[1:] - F[:-1]) / G.V_c[:, None, None, None]
    if return_walls:
        return adv, (nw_L, nw_R)
    return adv


# ----------------------------------------------------------------------------- force
def force(f, P: Problem):
    """Curvature term of Secs. II.B (cylinder) and II.C (sphere) with the matrices of Sec. III.B."""
    KRf = np.einsum("ab,cbjk->cajk", P.KR, f)
    K2f = np.einsum("ab,cibk->ciak", P.K2, f)
    pR = P.pR[None, :, None, None]
    p2 = P.p2[None, None, :, None]
    p3 = P.p3[None, None, None, :]
    kap = P.grid.kappa[:, None, None, None]
    if P.geometry == geo.CYL:
        return kap * (p2 * p2 * KRf - pR * K2f)
    K3f = np.einsum("ab,cija->cijb", P.K3.T, f)
    return 0.5 * kap * ((p2 * p2 + p3 * p3) * KRf - pR * (K2f + K3f))


# ----------------------------------------------------------------------------- RHS and RK3
def rhs(f, P: Problem, details=False):
    """L(f) = -advection - force + collision."""
    cl = closure(f, P)
    adv, walls = advection(f, P, return_walls=True)
    frc = force(f, P)
    col = collision_reduced(f, P, cl) if P.reduced else collision(f, P, cl)
    L = -adv - frc + col
    if details:
        return L, dict(closure=cl, adv=adv, force=frc, coll=col, n_wall=walls)
    return L


def rk3_step(f, P: Problem):
    """One SSP-RK3 step: f1 = f + dt L(f); f2 = 3/4 f + 1/4 (f1 + dt L(f1));
    f^{n+1} = 1/3 f + 2/3 (f2 + dt L(f2))."""
    dt = P.dt
    f1 = f + dt * rhs(f, P)
    f2 = 0.75 * f + 0.25 * (f1 + dt * rhs(f1, P))
    return f / 3.0 + 2.0 / 3.0 * (f2 + dt * rhs(f2, P))


def run(f, P: Problem, steps: int):
    for _ in range(steps):
        f = rk3_step(f, P)
    return f


# ----------------------------------------------------------------------------- initial states
def uniform_state(P: Problem, n0=None, T0=None):
    """Uniform equilibrium n0 g_R(0, T0) g_2(0, T0) g_3(0, T0), T0 = mean wall temperature (A15)."""
    n0 = P.n0 if n0 is None else n0
    T0 = 0.5 * (P.T_wall[0] + P.T_wall[1]) if T0 is None else T0
    gR = eq.g_half(P.pR, P.wR, P.alphaR, P.betaR, P.NR, 0.0, T0)
    g2 = eq.g_full(P.p2, P.w2, P.N2, 0.0, T0)
    g3 = np.array([1.0, T0]) if P.reduced else eq.g_full(P.p3, P.w3, P.N3, 0.0, T0)
    f = n0 * gR[:, None, None] * g2[None, :, None] * g3[None, None, :]
    return np.broadcast_to(f, P.shape).copy()


def shakhov_seed(P: Problem, n, u2, T, qR):
    """Warm-start populations from moment profiles on the cells:
    f = n g_R(0, T) g_2(u_2, T) g_3(0, T) [1 + (xi^2/(5T) - 1) xi_R q_R / (n T^2)]
    (the Shakhov factor of Sec. II with 1 - Pr replaced by 1, so that the seeded q_R is
    carried by the populations)."""
    gR = eq.g_half(P.pR, P.wR, P.alphaR, P.betaR, P.NR, np.zeros_like(T), T)
    g2 = eq.g_full(P.p2, P.w2, P.N2, u2, T)
    e = lambda a: a[:, None, None, None]
    if P.reduced:
        # the p_z-integrals against 1 and p_z^2 (xi^2 carries p_z^2 -> T, 3T; chi weighted by T)
        x0 = P.pR[None, :, None]
        xs = x0 ** 2 + (P.p2[None, None, :] - u2[:, None, None]) ** 2
        base = n[:, None, None] * gR[:, :, None] * g2[:, None, :]
        f = np.empty(base.shape + (2,))
        t = T[:, None, None]
        qf = x0 * (qR / (n * T * T))[:, None, None]
        f[..., 0] = base * (1.0 + ((xs + t) / (5.0 * t) - 1.0) * qf)
        f[..., 1] = t * base * (1.0 + ((xs + 3.0 * t) / (5.0 * t) - 1.0) * qf)
        return f
    g3 = eq.g_full(P.p3, P.w3, P.N3, np.zeros_like(T), T)
    p = momentum_axes(P)
    xi2 = p[0][None] ** 2 + (p[1][None] - e(u2)) ** 2 + p[2][None] ** 2
    fMB = e(n) * gR[:, :, None, None] * g2[:, None, :, None] * g3[:, None, None, :]
    return fMB * (1.0 + (xi2 / (5.0 * e(T)) - 1.0) * p[0][None] * e(qR) / e(n * T * T))


# ----------------------------------------------------------------------------- diagnostics
def total_mass(f, P: Problem):
    """sum_c V_c n_c (per unit angle, and per unit length for the cylinder)."""
    n = f[..., 0].sum((1, 2)) if P.reduced else f.sum((1, 2, 3))
    return float((P.grid.V_c * n).sum())


def moment_residual(m_old, m_new, K, scales):
    """max over {n, u_2, T, q_R} of ||M_new - M_old||_inf / (K max(||M_old||_inf, scale_M))
    (A11 reading: per-step relative change of the moment profiles over K steps)."""
    r = 0.0
    for key, s in zip(("n", "u2", "T", "qR"), scales):
        a, b = m_old[key], m_new[key]
        r = max(r, float(np.max(np.abs(b - a))) / (K * max(float(np.max(np.abs(a))), s)))
    return r


def profile_moments(f, P: Problem):
    m = moments(f, P)
    return {"n": m["n"], "u2": m["u"][:, 1], "T": m["T"], "qR": m["q"][:, 0]}
