"""Pins of the oracle's time step (Secs. II-III): conservation, steady uniform equilibrium,
mirror symmetry, a long-hand brute-force RHS on a tiny grid, and the analytic
Navier-Stokes Couette profile u_phi = A R + B/R (Sec. II macroscopic equations)."""
import math

import numpy as np
import pytest

from oracle import equilibrium as eq
from oracle import geometry as geo
from oracle import model
from oracle import solver as S
from paper_2403_15051_gb300 import workloads as wl


def _perturbed(P, seed=1, amp=0.05):
    return S.uniform_state(P) * wl.perturbation(P.shape, seed, amp)


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_mass_conserved_to_roundoff(g, beta):
    # needs N_a >= 3 on every axis: the Shakhov and J1 factors are cubic in xi (A5 reading)
    P = S.make_problem(g, 1.0, 2.5, 24, 4, 4, 5, eta0=0.15, Kn=0.1, beta=beta,
                       T_wall=(1.0, 1.2), u_wall=((0.2, 0.0) if g == geo.CYL else (0.0, 0.0)))
    f = _perturbed(P)
    m0 = S.total_mass(f, P)
    f = S.run(f, P, 20)
    assert abs(S.total_mass(f, P) - m0) / m0 < 1e-13


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_uniform_equilibrium_is_steady(g, beta):
    # walls at rest at T = 1 and chi from the local density: the uniform equilibrium is an
    # exact discrete steady state (advection, curvature force and wall terms cancel)
    P = S.make_problem(g, 1.0, 3.0, 20, 4, 4, 4, eta0=0.2, Kn=0.1, beta=beta, chi_model=S.SET_LOCAL)
    f = S.uniform_state(P)
    L = S.rhs(f, P)
    assert np.max(np.abs(L)) < 1e-12 * np.max(np.abs(f)) / P.dt * P.dt  # relative to f per unit time
    g1 = S.run(f, P, 5)
    assert np.max(np.abs(g1 - f)) <= 1e-13 * np.max(np.abs(f))


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
def test_collision_and_force_conserve_mass_per_cell(g):
    P = S.make_problem(g, 1.0, 2.0, 16, 4, 4, 4, eta0=0.2, Kn=0.05, T_wall=(1.0, 1.3))
    f = _perturbed(P, seed=3, amp=0.1)
    _, d = S.rhs(f, P, details=True)
    scale = np.abs(d["coll"]).sum((1, 2, 3))
    assert np.all(np.abs(d["coll"].sum((1, 2, 3))) <= 1e-13 * scale)
    scale = np.abs(d["force"]).sum((1, 2, 3))
    assert np.all(np.abs(d["force"].sum((1, 2, 3))) <= 1e-13 * scale)


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
@pytest.mark.parametrize("chi_model", [S.SET_LOCAL, S.RET_FM])
def test_collision_momentum_and_energy_moments(g, chi_model):
    """Gaussian moments of the collision term (Eqs. shakhov, j1) on a perturbed state.  The
    Shakhov part conserves momentum and energy; the first-order Enskog term J1 transfers
    momentum -P_c X along R only (P_c = b rho chi n T, the non-ideal part of the pressure;
    X = d ln(n^2 chi T)/dR, so -grad P_c for the local chi) and does the work -P_c div u (the
    Y term and the (zeta^2 - 5/2) div u term carry neither).  The degree-5 energy moment of the
    Shakhov correction is exact from Q = 6 (expansion order 5) on."""
    P = S.make_problem(g, 1.0, 2.0, 16, 6, 6, 6, eta0=0.2, Kn=0.05, T_wall=(1.0, 1.3), chi_model=chi_model,
                       u_wall=((0.2, 0.0) if g == geo.CYL else (0.0, 0.0)))
    f = _perturbed(P, seed=3, amp=0.1)
    _, d = S.rhs(f, P, details=True)
    C, cl = d["coll"], d["closure"]
    ax = (1, 2, 3)
    p = S.momentum_axes(P)
    u = cl["u"]
    xi = [p[a][None] - u[:, a][:, None, None, None] for a in range(3)]
    Pc = cl["br"] * cl["chi"] * cl["n"] * cl["T"]
    scale = np.abs(C).sum(ax)
    mom = [(C * p[a]).sum(ax) for a in range(3)]
    energy = (C * 0.5 * (xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2)).sum(ax)
    assert np.max(np.abs(Pc * cl["X"]) / scale) > 0.1 and np.max(np.abs(Pc * cl["div"]) / scale) > 0.1
    assert np.all(np.abs(mom[0] + Pc * cl["X"]) <= 1e-13 * scale)
    assert np.all(np.abs(mom[1]) <= 1e-13 * scale) and np.all(np.abs(mom[2]) <= 1e-13 * scale)
    assert np.all(np.abs(energy + Pc * cl["div"]) <= 1e-13 * scale)


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
@pytest.mark.parametrize("Q", [3, 5])
def test_force_momentum_and_energy_moments(g, Q):
    """Momentum moments of the curvature term (Secs. II.B, II.C), integrated by parts in momentum
    space: with kappa = (A_+ - A_-)/V (1/R on the cylinder, 2/R on the sphere) the force term F
    (entering the RHS as -F) has radial moment -kappa M_22 (cylinder) or -kappa (M_22 + M_33)/2
    (sphere), the centrifugal pressure, and tangential moments kappa M_R2 (cylinder) or
    kappa M_R2 / 2 and kappa M_R3 / 2 (sphere), the curvature part of the angular-momentum
    balance; its energy moment is zero.  This holds on any nodal state, since the derivative
    matrices are exact on the polynomials involved (stretched grid, perturbed state)."""
    P = S.make_problem(g, 1.0, 2.0, 16, Q, Q, Q, eta0=0.2, Kn=0.05, beta=1.0, T_wall=(1.0, 1.3),
                       u_wall=((0.2, 0.0) if g == geo.CYL else (0.0, 0.0)))
    f = _perturbed(P, seed=3, amp=0.1)
    F = S.force(f, P)
    ax = (1, 2, 3)
    p = S.momentum_axes(P)
    k = P.grid.kappa
    M = lambda a, b: (f * p[a] * p[b]).sum(ax)
    mom = [(F * p[a]).sum(ax) for a in range(3)]
    energy = (F * 0.5 * (p[0] ** 2 + p[1] ** 2 + p[2] ** 2)).sum(ax)
    if g == geo.CYL:
        want = [-k * M(1, 1), k * M(0, 1), np.zeros_like(k)]
    else:
        want = [-0.5 * k * (M(1, 1) + M(2, 2)), 0.5 * k * M(0, 1), 0.5 * k * M(0, 2)]
    scale = np.abs(F).sum(ax)
    assert np.min(np.abs(want[1]) / scale) > 1e-4
    for a in range(3):
        assert np.all(np.abs(mom[a] - want[a]) <= 1e-13 * scale), a
    assert np.all(np.abs(energy) <= 1e-13 * scale)


def test_mirror_symmetry_of_wall_speed():
    # u_w -> -u_w flips u_phi and q_phi and leaves n, T, q_R unchanged
    kw = dict(eta0=0.1, Kn=0.1)
    Pa = S.make_problem(geo.CYL, 1.0, 2.0, 16, 4, 4, 4, u_wall=(0.2, 0.0), **kw)
    Pb = S.make_problem(geo.CYL, 1.0, 2.0, 16, 4, 4, 4, u_wall=(-0.2, 0.0), **kw)
    fa = S.run(S.uniform_state(Pa), Pa, 30)
    fb = S.run(S.uniform_state(Pb), Pb, 30)
    ma, mb = S.moments(fa, Pa), S.moments(fb, Pb)
    assert np.allclose(ma["n"], mb["n"], rtol=1e-12)
    assert np.allclose(ma["T"], mb["T"], rtol=1e-12)
    assert np.allclose(ma["q"][:, 0], mb["q"][:, 0], atol=1e-11 * np.abs(ma["q"]).max())
    assert np.allclose(ma["u"][:, 1], -mb["u"][:, 1], atol=1e-13)
    assert np.allclose(ma["q"][:, 1], -mb["q"][:, 1], atol=1e-11 * np.abs(ma["q"]).max())
    assert np.abs(ma["u"][:, 1]).max() > 1e-3


# ----------------------------------------------------------------------------- brute force
def _weno_scalar(a, b, c, d, e, eps=1e-6):
    # Jiang-Shu fifth-order reconstruction at the right face of c, upwind from the left
    s0 = 13 / 12 * (a - 2 * b + c) ** 2 + 1 / 4 * (a - 4 * b + 3 * c) ** 2
    s1 = 13 / 12 * (b - 2 * c + d) ** 2 + 1 / 4 * (b - d) ** 2
    s2 = 13 / 12 * (c - 2 * d + e) ** 2 + 1 / 4 * (3 * c - 4 * d + e) ** 2
    w = [0.1 / (eps + s0) ** 2, 0.6 / (eps + s1) ** 2, 0.3 / (eps + s2) ** 2]
    r = [(2 * a - 7 * b + 11 * c) / 6, (-b + 5 * c + 2 * d) / 6, (2 * c + 5 * d - e) / 6]
    return sum(wi * ri for wi, ri in zip(w, r)) / sum(w)


def longhand_rhs(f, P):
    """The same equations as oracle.solver.rhs, evaluated cell by cell and momentum by
    momentum with scalar loops (no array broadcasting)."""
    G = P.grid
    N, nR, n2, n3 = f.shape
    pa = [P.pR, P.p2, P.p3]
    wgt = lambda i, j, k: P.wR[i] * P.w2[j] * P.w3[k]
    # moments
    n = np.zeros(N); u = np.zeros((N, 3)); T = np.zeros(N); q = np.zeros((N, 3))
    for c in range(N):
        s0 = 0.0; s1 = np.zeros(3); s2 = np.zeros((3, 3)); s3 = np.zeros(3)
        for i in range(nR):
            for j in range(n2):
                for k in range(n3):
                    p = np.array([pa[0][i], pa[1][j], pa[2][k]])
                    v = f[c, i, j, k]
                    s0 += v; s1 += v * p; s2 += v * np.outer(p, p); s3 += v * (p @ p) * p
        n[c] = s0; u[c] = s1 / s0
        T[c] = (np.trace(s2) - s0 * u[c] @ u[c]) / (3 * s0)
        for i in range(nR):
            for j in range(n2):
                for k in range(n3):
                    xi = np.array([pa[0][i], pa[1][j], pa[2][k]]) - u[c]
                    q[c] += 0.5 * f[c, i, j, k] * (xi @ xi) * xi
    # closure
    nbar = np.array([sum(P.W[c, d] * n[d] for d in range(N)) for c in range(N)])
    chi = np.array([model.chi_set(math.pi * P.sigma ** 3 * nb / 6) for nb in nbar])
    br = 2 * math.pi / 3 * P.sigma ** 3 * n
    Pr = np.array([model.prandtl(n[c], chi[c], P.sigma) for c in range(N)])
    tau = np.array([model.relaxation_time(n[c], T[c], chi[c], P.sigma) for c in range(N)])
    X, Y = S.d_dR(np.log(n * n * chi * T), G), S.d_dR(np.log(T), G)
    du = [S.d_dR(u[:, a], G) for a in range(3)]
    out = np.zeros_like(f)
    for c in range(N):
        R = G.R_c[c]
        Sab = np.zeros((3, 3))
        Sab[0, 0] = du[0][c]
        Sab[0, 1] = Sab[1, 0] = 0.5 * (du[1][c] - u[c, 1] / R)
        if P.geometry == geo.CYL:
            Sab[1, 1] = u[c, 0] / R
            Sab[0, 2] = Sab[2, 0] = 0.5 * du[2][c]
            div = du[0][c] + u[c, 0] / R
        else:
            Sab[1, 1] = Sab[2, 2] = u[c, 0] / R
            Sab[0, 2] = Sab[2, 0] = 0.5 * (du[2][c] - u[c, 2] / R)
            div = du[0][c] + 2 * u[c, 0] / R
        gR = eq.g_half(P.pR, P.wR, P.alphaR, P.betaR, P.NR, u[c, 0], T[c])
        g2 = eq.g_full(P.p2, P.w2, P.N2, u[c, 1], T[c])
        g3 = eq.g_full(P.p3, P.w3, P.N3, u[c, 2], T[c])
        for i in range(nR):
            for j in range(n2):
                for k in range(n3):
                    xi = np.array([pa[0][i], pa[1][j], pa[2][k]]) - u[c]
                    x2 = xi @ xi
                    fmb = n[c] * gR[i] * g2[j] * g3[k]
                    fs = fmb * (1 + (1 - Pr[c]) / (n[c] * T[c] ** 2) * (x2 / (5 * T[c]) - 1) * (xi @ q[c]))
                    z2 = x2 / (2 * T[c])
                    strain = sum(xi[a] * xi[b] * Sab[a, b] for a in range(3) for b in range(3)) / T[c]
                    j1 = -br[c] * chi[c] * fmb * (xi[0] * (X[c] + 0.6 * (z2 - 2.5) * Y[c])
                                                   + 0.4 * (strain + (z2 - 2.5) * div))
                    out[c, i, j, k] += -(f[c, i, j, k] - fs) / tau[c] + j1
                    # force
                    KRf = sum(P.KR[i, a] * f[c, a, j, k] for a in range(nR))
                    K2f = sum(P.K2[j, b] * f[c, i, b, k] for b in range(n2))
                    if P.geometry == geo.CYL:
                        frc = G.kappa[c] * (pa[1][j] ** 2 * KRf - pa[0][i] * K2f)
                    else:
                        K3f = sum(P.K3[k, b] * f[c, i, j, b] for b in range(n3))
                        frc = 0.5 * G.kappa[c] * ((pa[1][j] ** 2 + pa[2][k] ** 2) * KRf - pa[0][i] * (K2f + K3f))
                    out[c, i, j, k] -= frc
    # advection, momentum by momentum
    gw = S.wall_maxwellians(P)
    vhat = {}
    for i in range(nR):
        for j in range(n2):
            for k in range(n3):
                w = wgt(i, j, k)
                v = [f[c, i, j, k] / w for c in range(N)]
                ext = {c: v[c] for c in range(N)}
                ext[-1] = 4 * v[0] - 6 * v[1] + 4 * v[2] - v[3]
                ext[-2] = 10 * v[0] - 20 * v[1] + 15 * v[2] - 4 * v[3]
                ext[N] = 4 * v[N - 1] - 6 * v[N - 2] + 4 * v[N - 3] - v[N - 4]
                ext[N + 1] = 10 * v[N - 1] - 20 * v[N - 2] + 15 * v[N - 3] - 4 * v[N - 4]
                vhat[(i, j, k)] = (_weno_scalar(ext[2], ext[1], ext[0], ext[-1], ext[-2]),
                                   _weno_scalar(ext[N - 3], ext[N - 2], ext[N - 1], ext[N], ext[N + 1]), ext)
    outL = sum(abs(pa[0][i]) * wgt(i, j, k) * vhat[(i, j, k)][0]
               for i in range(nR) for j in range(n2) for k in range(n3) if pa[0][i] < 0)
    inL = sum(pa[0][i] * gw[0][i, j, k] for i in range(nR) for j in range(n2) for k in range(n3) if pa[0][i] > 0)
    outR = sum(pa[0][i] * wgt(i, j, k) * vhat[(i, j, k)][1]
               for i in range(nR) for j in range(n2) for k in range(n3) if pa[0][i] > 0)
    inR = sum(abs(pa[0][i]) * gw[1][i, j, k] for i in range(nR) for j in range(n2) for k in range(n3) if pa[0][i] < 0)
    nwL, nwR = outL / inL, outR / inR
    for i in range(nR):
        for j in range(n2):
            for k in range(n3):
                w = wgt(i, j, k)
                vl, vr, ext = vhat[(i, j, k)]
                p = pa[0][i]
                if p > 0:
                    ext[-1] = ext[-2] = nwL * gw[0][i, j, k] / w
                else:
                    ext[N] = ext[N + 1] = nwR * gw[1][i, j, k] / w
                F = np.zeros(N + 1)
                for fc in range(N + 1):
                    if fc == 0:
                        val = nwL * gw[0][i, j, k] if p > 0 else w * vl
                    elif fc == N:
                        val = w * vr if p > 0 else nwR * gw[1][i, j, k]
                    elif p > 0:
                        val = w * _weno_scalar(ext[fc - 3], ext[fc - 2], ext[fc - 1], ext[fc], ext[fc + 1])
                    else:
                        val = w * _weno_scalar(ext[fc + 2], ext[fc + 1], ext[fc], ext[fc - 1], ext[fc - 2])
                    F[fc] = G.A_f[fc] * p * val
                for c in range(N):
                    out[c, i, j, k] -= (F[c + 1] - F[c]) / G.V_c[c]
    return out


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
def test_vectorised_rhs_matches_longhand_loops(g):
    P = S.make_problem(g, 1.0, 2.0, 7, 2, 3, 2, eta0=0.2, Kn=0.3, beta=0.7, T_wall=(1.0, 1.25),
                       u_wall=((0.15, 0.0) if g == geo.CYL else (0.0, 0.0)))
    f = _perturbed(P, seed=7, amp=0.1)
    a = S.rhs(f, P)
    b = longhand_rhs(f, P)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-12 * np.abs(b).max())


# ----------------------------------------------------------------------------- physics
@pytest.mark.slow
def test_couette_profile_is_A_R_plus_B_over_R_in_the_dilute_small_Kn_limit():
    """Navier-Stokes steady cylindrical Couette flow has u_phi = A R + B / R (Sec. II
    macroscopic equations with the Newton stress law); a dilute gas at Kn = 0.05 must follow
    that form in the bulk, with A and B within slip corrections of the no-slip values."""
    R1, R2, uw = 1.0, 2.0, 0.05
    P = S.make_problem(geo.CYL, R1, R2, 24, 4, 4, 4, eta0=0.001, Kn=0.05, u_wall=(uw, 0.0))
    A0 = uw * R1 / (R1 ** 2 - R2 ** 2)
    B0 = uw * R1 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
    Rc = P.grid.R_c
    n = np.full(P.grid.N, P.n0)
    f = S.shakhov_seed(P, n, A0 * Rc + B0 / Rc, np.ones_like(Rc), np.zeros_like(Rc))
    steps = int(round(12.0 / P.dt))
    f = S.run(f, P, steps)
    last = S.profile_moments(f, P)
    f = S.run(f, P, 100)
    assert S.moment_residual(last, S.profile_moments(f, P), 100, (P.n0, 1, 1, P.n0)) < 1e-6
    uphi = S.moments(f, P)["u"][:, 1]
    bulk = slice(4, -4)
    M = np.stack([Rc, 1 / Rc], 1)[bulk]
    (A, B), *_ = np.linalg.lstsq(M, uphi[bulk], rcond=None)
    fit_res = np.max(np.abs(M @ np.array([A, B]) - uphi[bulk]))
    M1 = np.stack([Rc, np.ones_like(Rc)], 1)[bulk]
    c1, *_ = np.linalg.lstsq(M1, uphi[bulk], rcond=None)
    lin_res = np.max(np.abs(M1 @ c1 - uphi[bulk]))
    assert fit_res < 2e-3 * uw
    assert lin_res > 5 * fit_res  # the curvature of the profile is resolved
    assert A == pytest.approx(A0, rel=0.25) and B == pytest.approx(B0, rel=0.25)
    # the emergent shear viscosity: away from the Knudsen layers the kinetic shear stress is the
    # Newton law P_R2 = -mu R d(u_phi/R)/dR with mu = tau P_i from the Eq. viscosity coefficient
    m = S.moments(f, P)
    chi = model.chi_set(model.eta_of_n(m["n"], P.sigma))
    mu = model.viscosity(m["n"], m["T"], chi, P.sigma)
    ratio = (m["P01"] / (-mu * (S.d_dR(uphi, P.grid) - uphi / Rc)))[8:16]
    assert np.all(np.abs(ratio - 1) < 0.01), ratio
    # torque balance: J1 carries no phi-momentum, so R^2 P_R2 is constant across the gap
    R2P = (Rc ** 2 * m["P01"])[3:-3]
    assert (R2P.max() - R2P.min()) / abs(R2P.mean()) < 0.01


@pytest.mark.slow
def test_fourier_flow_radial_heat_flux_constant_times_R_squared():
    """Steady Fourier flow between concentric spheres: with the gas at rest the energy balance
    reduces to d(R^2 q_R)/dR = 0, so R^2 q_R is constant across the gap (Sec. IV.B, geometry
    comparison) and q_R falls off as R^-2.  A spherical metric factor taken as the cylinder's (one
    power of R) would give R q_R constant instead, which this rejects.  The first and last three
    cells hold the Knudsen layers and the one-sided wall stencils and are left out."""
    P = S.make_problem(geo.SPH, 1.0, 2.0, 24, 4, 4, 4, eta0=0.1, Kn=0.1, T_wall=(1.1, 0.9))
    f = S.uniform_state(P)
    f = S.run(f, P, int(round(12.0 / P.dt)))
    m = S.moments(f, P)
    R, qR = P.grid.R_c[3:-3], m["q"][3:-3, 0]
    assert np.all(qR > 0)
    R2q, Rq = R ** 2 * qR, R * qR
    assert (R2q.max() - R2q.min()) / R2q.mean() < 0.01
    assert (Rq.max() - Rq.min()) / Rq.mean() > 0.2
    slope = np.polyfit(np.log(R), np.log(qR), 1)[0]
    assert slope == pytest.approx(-2.0, abs=0.02)


@pytest.mark.slow
def test_fourier_flow_conductivity_in_the_dilute_small_Kn_limit():
    """The emergent thermal conductivity of the Shakhov model (Sec. II): in a dilute gas at
    Kn = 0.05 the steady radial heat flux between cylinders follows Fourier's law q_R = -lambda
    dT/dR with lambda = (5/2) tau P_i / Pr (Eq. viscosity, second line; Pr -> 2/3) in the cells
    away from the Knudsen layers.  A Shakhov correction dropped (Pr = 1) or of the wrong sign
    changes lambda by a third or more."""
    P = S.make_problem(geo.CYL, 1.0, 2.0, 24, 4, 4, 4, eta0=0.001, Kn=0.05, T_wall=(1.1, 0.9))
    f = S.run(S.uniform_state(P), P, int(round(12.0 / P.dt)))
    m = S.moments(f, P)
    chi = model.chi_set(model.eta_of_n(m["n"], P.sigma))
    lam = model.conductivity(m["n"], m["T"], chi, P.sigma)
    ratio = (m["q"][:, 0] / (-lam * S.d_dR(m["T"], P.grid)))[8:16]
    assert np.all(np.abs(ratio - 1) < 0.015), ratio


# ----------------------------------------------------------------------------- convergence orders
def _observed_orders(errors):
    e = np.asarray(errors)
    return np.log2(e[:-1] / e[1:])


@pytest.mark.parametrize("upwind", [+1, -1])
def test_weno5_flux_difference_converges_at_fifth_order(upwind):
    """Finite-difference WENO5-JS on point values (Sec. III.A, A8 reading): the difference of the
    reconstructed face values over h approximates the derivative to O(h^5) on a smooth profile
    without critical points, upwind from either side."""
    def err(N):
        h = 1.0 / N
        x = (np.arange(-3, N + 3) + 0.5) * h
        g = np.exp(x) + 0.5 * np.sin(3 * x)
        i = np.arange(3, N + 3)
        if upwind > 0:
            right = S.weno5(g[i - 2], g[i - 1], g[i], g[i + 1], g[i + 2])
            left = S.weno5(g[i - 3], g[i - 2], g[i - 1], g[i], g[i + 1])
        else:
            right = S.weno5(g[i + 3], g[i + 2], g[i + 1], g[i], g[i - 1])
            left = S.weno5(g[i + 2], g[i + 1], g[i], g[i - 1], g[i - 2])
        exact = np.exp(x[i]) + 1.5 * np.cos(3 * x[i])
        return np.max(np.abs((right - left) / h - exact))
    orders = _observed_orders([err(N) for N in (20, 40, 80, 160)])
    assert np.all(orders[1:] > 4.7), orders


@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_radial_gradients_converge_at_fourth_order(beta):
    """The closure's radial derivative (fourth-order central differences in the mapped coordinate,
    one-sided five-point stencils in the two cells by each wall; Sec. III.A, A9 reading) on a
    uniform and a stretched grid: O(h^4) in the max norm over every cell."""
    def err(N):
        G = geo.make_grid(geo.CYL, 1.0, 2.0, 0.01, N, beta)
        R = G.R_c
        exact = np.exp(R) * (np.sin(2 * R) + 2 * np.cos(2 * R))
        return np.max(np.abs(S.d_dR(np.exp(R) * np.sin(2 * R), G) - exact))
    orders = _observed_orders([err(N) for N in (16, 32, 64, 128)])
    assert np.all(orders > 3.8), orders


@pytest.mark.parametrize("g,horizon", [(geo.CYL, 10), (geo.SPH, 20)])
def test_ssp_rk3_converges_at_third_order_in_time(g, horizon):
    """The time integrator (Sec. III, SSP-RK3) on a smooth transient of the semi-discrete system:
    halving the step divides the difference between successive solutions at a fixed time by 2^3.
    Mass conservation and steady states do not see the stage coefficients; this does."""
    import dataclasses
    P0 = S.make_problem(g, 1.0, 2.0, 16, 3, 3, 3, eta0=0.1, Kn=0.3, T_wall=(1.0, 1.2),
                        u_wall=((0.1, 0.0) if g == geo.CYL else (0.0, 0.0)))
    R = P0.grid.R_c
    x = (R - R[0]) / (R[-1] - R[0])
    uphi = 0.05 * np.sin(np.pi * x) if g == geo.CYL else np.zeros_like(x)
    f0 = S.shakhov_seed(P0, P0.n0 * (1 + 0.05 * np.cos(np.pi * x)), uphi, 1 + 0.1 * x, 0.01 * np.sin(np.pi * x))
    f = {k: S.run(f0, dataclasses.replace(P0, dt=P0.dt / k), horizon * k) for k in (1, 2, 4, 8)}
    e = [np.max(np.abs(f[k] - f[2 * k])) for k in (1, 2, 4)]
    ratios = [e[0] / e[1], e[1] / e[2]]
    assert all(6.0 < r < 11.0 for r in ratios), ratios


@pytest.mark.slow
def test_dense_fourier_flow_radial_momentum_balance():
    """Steady dense-gas Fourier flow between cylinders (eta0 = 0.2, RET-FM chi).  The energy balance
    makes R q_R constant across the gap (Sec. IV.B, geometry comparison: q^R R = const), heat
    flowing outwards from the hot inner wall.  The gas is at rest,
    so the first moment of the kinetic equation reduces to dP_RR/dR + (P_RR - P_22)/R = -P_c X,
    the kinetic pressure gradient and the curvature of the stress balanced by the momentum that J1
    transfers (P_c = b rho chi n T, X = d ln(n^2 chi T)/dR; Eq. j1, Sec. II.B).  Away from the
    Knudsen layers the balance holds to 3% of P_c X (discretisation); a gradient term taken
    without the n^2, chi or T factor breaks it by 60% or more."""
    P = S.make_problem(geo.CYL, 1.0, 2.0, 24, 4, 4, 4, eta0=0.2, Kn=0.1, T_wall=(1.2, 0.8))
    f = S.run(S.uniform_state(P), P, int(round(12.0 / P.dt)))
    n, u, T, q, M2 = S.macroscopic(S.raw_sums(f, P))
    Rq = P.grid.R_c * q[:, 0]
    assert np.all(Rq > 0) and (Rq.max() - Rq.min()) / Rq.mean() < 0.02
    P_RR = M2[:, 0, 0] - n * u[:, 0] ** 2
    P_22 = M2[:, 1, 1] - n * u[:, 1] ** 2
    chi = model.chi_set(model.eta_of_n(P.W @ n, P.sigma))
    Pc = model.b_rho(n, P.sigma) * chi * n * T
    X = S.d_dR(np.log(n * n * chi * T), P.grid)
    balance = S.d_dR(P_RR, P.grid) + (P_RR - P_22) / P.grid.R_c + Pc * X
    scale = np.max(np.abs(Pc * X)[3:-3])
    assert scale > 0.1 * np.max(np.abs(S.d_dR(P_RR, P.grid))[3:-3])
    assert np.max(np.abs(balance[3:-3])) < 0.03 * scale


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
def test_diffuse_walls_pull_the_adjacent_gas_toward_their_state(g):
    """Diffuse reflection (Sec. IV walls): particles leave each wall with the wall's Maxwellian, so
    within 20 steps from rest at T = 1 the gas next to the hot inner wall (T = 1.2) warms and the
    gas next to the cold outer wall (T = 0.8) cools, and next to the moving inner cylinder wall
    (u_2 = 0.1) it is dragged along the wall's direction but not past the wall's speed, while the
    gas at the resting outer wall is not yet moving."""
    P = S.make_problem(g, 1.0, 2.0, 16, 4, 4, 4, eta0=0.1, Kn=0.1, T_wall=(1.2, 0.8),
                       u_wall=((0.1, 0.0) if g == geo.CYL else (0.0, 0.0)))
    m = S.moments(S.run(S.uniform_state(P), P, 20), P)
    assert m["T"][0] > 1.03 and m["T"][-1] < 0.97
    assert np.all(np.diff(m["T"]) < 0)
    if g == geo.CYL:
        assert 0.01 < m["u"][0, 1] < 0.1 and abs(m["u"][-1, 1]) < 1e-4
        assert np.max(np.abs(m["u"][:, 2])) < 1e-12


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
def test_shakhov_seed_reproduces_its_moment_profiles(g):
    """The warm-start seed f = n g_R(0,T) g_2(u_2,T) g_3(0,T) [1 + (xi^2/(5T) - 1) xi_R q_R/(n T^2)]
    carries the profiles it is built from: its quadrature moments (Eq. macro_def) are n, u_2, T
    and q_R again, with u_R = u_3 = 0, to round-off.  The Shakhov factor is odd in xi_R, so it
    leaves n, u and T alone, and its heat flux is q_R <(xi^2/(5T) - 1) xi_R^2 xi^2>/(2T^2) =
    q_R (35 T^3/(5T) - 5 T^2)/(2 T^2) = q_R, Gaussian moments of degree 6 in xi_R and 4 in xi_2,
    xi_3: the expansion orders must reach them (N_R >= 6, N_2, N_3 >= 4; here 7, 5, 5)."""
    P = S.make_problem(g, 1.0, 2.0, 12, 8, 6, 6, eta0=0.1, Kn=0.1)
    x = (np.arange(12) + 0.5) / 12
    n = P.n0 * (1.0 + 0.2 * np.sin(2.0 * x))
    u2 = 0.25 * np.cos(3.0 * x)
    T = 0.9 + 0.3 * x
    qR = 0.03 * P.n0 * (x - 0.4)
    m = S.moments(S.shakhov_seed(P, n, u2, T, qR), P)
    assert np.allclose(m["n"], n, rtol=1e-13, atol=0)
    assert np.max(np.abs(m["u"][:, 1] - u2)) < 1e-13
    assert np.max(np.abs(m["u"][:, 0])) < 1e-13 and np.max(np.abs(m["u"][:, 2])) < 1e-13
    assert np.allclose(m["T"], T, rtol=1e-13, atol=0)
    assert np.max(np.abs(m["q"][:, 0] - qR)) < 1e-12 * P.n0
    # with no heat flux and constant profiles it is the uniform equilibrium
    f_u = S.shakhov_seed(P, np.full(12, P.n0), np.zeros(12), np.full(12, 1.1), np.zeros(12))
    assert np.max(np.abs(f_u - S.uniform_state(P, T0=1.1))) <= 1e-13 * np.max(f_u)


def test_moment_residual_on_a_hand_computed_two_cell_case():
    """r = max over (n, u_2, T, q_R) of max_c |M_new - M_old| / (K max(max_c |M_old|, scale)),
    worked by hand for two cells and K = 3 steps:
      n:   max|dn| = |4.6 - 4.0| = 0.6, max|n_old| = 4 > scale 1      -> 0.6 / (3 * 4)   = 0.05
      u_2: max|du| = |-0.24 + 0.3| = 0.06, max|u_old| = 0.3 < scale 1 -> 0.06 / (3 * 1)  = 0.02
      T:   unchanged                                                   -> 0
      q_R: max|dq| = 1e-3, max|q_old| = 0 < scale 0.005               -> 1e-3 / 0.015   = 0.0667
    so r = 1/15 (the heat flux); with its scale raised to 0.05, r = 0.05 (the density), and with
    the density scale raised to 10 as well, r = 0.02 (the velocity)."""
    old = {"n": np.array([2.0, 4.0]), "u2": np.array([0.1, -0.3]), "T": np.array([1.0, 1.5]),
           "qR": np.array([0.0, 0.0])}
    new = {"n": np.array([2.3, 4.6]), "u2": np.array([0.1, -0.24]), "T": np.array([1.0, 1.5]),
           "qR": np.array([1e-3, 0.0])}
    assert S.moment_residual(old, new, 3, (1.0, 1.0, 1.0, 0.005)) == pytest.approx(1.0 / 15.0, rel=1e-14)
    assert S.moment_residual(old, new, 3, (1.0, 1.0, 1.0, 0.05)) == pytest.approx(0.05, rel=1e-14)
    assert S.moment_residual(old, new, 3, (10.0, 1.0, 1.0, 0.05)) == pytest.approx(0.02, rel=1e-14)
    assert S.moment_residual(old, old, 3, (1.0, 1.0, 1.0, 1.0)) == 0.0
