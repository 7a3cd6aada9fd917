"""Radial grid, finite-volume metric factors and Fischer-Methfessel weights.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Computational domain [R_L + sigma/2, R_R - sigma/2] (Sec. IV, first paragraph).
* N cells on the mapped coordinate s in [0, 1]; R(s) uniform, or tanh-stretched
  R(s) = R_L^c + L_c [1 + tanh(beta (2s - 1)) / tanh(beta)] / 2 (finer near both walls).
* Conservative advection (Sec. II.B/C): face areas A = R (cylinder) or r^2 (sphere),
  cell volumes V = int A dR, curvature factor kappa_i = (A_{i+1/2} - A_{i-1/2}) / V_i.
* Fischer-Methfessel average (Eq. fm): W_ij = 3/(4 pi sigma^3) |ball(sigma, x_i) cap shell_j|,
  with n = 0 outside the computational domain.  Sphere: lens volume of App. A; cylinder:
  the ball/cylinder intersection volume as an integral over z of the circle-circle lens area.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CYL = 0
SPH = 1


@dataclass
class Grid:
    geometry: int
    N: int
    s_c: np.ndarray      # (N,) mapped cell-centre coordinates
    R_c: np.ndarray      # (N,) cell-centre radii R(s_c)
    R_f: np.ndarray      # (N+1,) face radii R(k/N)
    dRds_c: np.ndarray   # (N,) dR/ds at the cell centres
    A_f: np.ndarray      # (N+1,) face areas per unit angle
    V_c: np.ndarray      # (N,) cell volumes per unit angle
    kappa: np.ndarray    # (N,) (A_+ - A_-) / V
    ds: float


def radius_map(s, RcL, Lc, beta):
    s = np.asarray(s, dtype=np.float64)
    if beta == 0.0:
        return RcL + Lc * s, Lc * np.ones_like(s)
    t = math.tanh(beta)
    R = RcL + 0.5 * Lc * (1.0 + np.tanh(beta * (2.0 * s - 1.0)) / t)
    dR = Lc * beta / np.cosh(beta * (2.0 * s - 1.0)) ** 2 / t
    return R, dR


def make_grid(geometry: int, R_L: float, R_R: float, sigma: float, N: int, beta: float = 0.0) -> Grid:
    """Grid over the computational domain [R_L + sigma/2, R_R - sigma/2]."""
    RcL = R_L + 0.5 * sigma
    Lc = (R_R - R_L) - sigma
    s_f = np.arange(N + 1) / N
    s_c = (np.arange(N) + 0.5) / N
    R_f, _ = radius_map(s_f, RcL, Lc, beta)
    R_c, dRds = radius_map(s_c, RcL, Lc, beta)
    if geometry == CYL:
        A_f = R_f.copy()
        V_c = 0.5 * (R_f[1:] ** 2 - R_f[:-1] ** 2)
    else:
        A_f = R_f ** 2
        V_c = (R_f[1:] ** 3 - R_f[:-1] ** 3) / 3.0
    kappa = (A_f[1:] - A_f[:-1]) / V_c
    return Grid(geometry, N, s_c, R_c, R_f, dRds, A_f, V_c, kappa, 1.0 / N)


# ----------------------------------------------------------------------------- FM weights
def lens_volume(r1, r2, d):
    """Volume common to two balls of radii r1, r2 whose centres are d apart (App. A),
    including the disjoint and nested cases."""
    r1, r2, d = np.broadcast_arrays(np.asarray(r1, float), np.asarray(r2, float), np.asarray(d, float))
    out = np.zeros(d.shape)
    rmin = np.minimum(r1, r2)
    nested = d <= np.abs(r1 - r2)
    out[nested] = 4.0 / 3.0 * math.pi * rmin[nested] ** 3
    part = (~nested) & (d < r1 + r2)
    dd, a, b = d[part], r1[part], r2[part]
    out[part] = math.pi * (a + b - dd) ** 2 * (dd * dd + 2 * dd * b - 3 * b * b + 2 * dd * a + 6 * a * b - 3 * a * a) / (12.0 * dd)
    return out


def circle_lens_area(r, d, Rp):
    """Area common to a disc of radius r centred at distance d from the origin and the disc
    of radius Rp centred at the origin (textbook circle-circle intersection)."""
    r, d, Rp = np.broadcast_arrays(np.asarray(r, float), np.asarray(d, float), np.asarray(Rp, float))
    out = np.zeros(r.shape)
    nested = d <= np.abs(Rp - r)
    out[nested] = math.pi * np.minimum(r, Rp)[nested] ** 2
    part = (~nested) & (d < r + Rp) & (r > 0)
    rr, dd, RR = r[part], d[part], Rp[part]
    c1 = np.clip((dd * dd + rr * rr - RR * RR) / (2 * dd * rr), -1.0, 1.0)
    c2 = np.clip((dd * dd + RR * RR - rr * rr) / (2 * dd * RR), -1.0, 1.0)
    k = (-dd + rr + RR) * (dd + rr - RR) * (dd - rr + RR) * (dd + rr + RR)
    out[part] = rr * rr * np.arccos(c1) + RR * RR * np.arccos(c2) - 0.5 * np.sqrt(np.maximum(k, 0.0))
    return out


_GL_CACHE = {}


def _gauss_legendre01(n):
    if n not in _GL_CACHE:
        x, w = np.polynomial.legendre.leggauss(n)
        _GL_CACHE[n] = (0.5 * (x + 1.0), 0.5 * w)
    return _GL_CACHE[n]


def ball_cylinder_volume(sigma, d, Rp, n_gl: int = 64):
    """|ball(radius sigma, centre at distance d from the axis) cap {rho < Rp}|
    = int_{-sigma}^{sigma} A(sqrt(sigma^2 - z^2), d, Rp) dz.

    With z = sigma sin t the integrand is smooth except where the disc radius
    sigma cos t crosses |Rp - d| or Rp + d; the t range [0, pi/2] is split there and each
    piece is integrated by Gauss-Legendre after the map t = a + (b - a)(1 - cos(pi u))/2,
    which absorbs the (r - r_b)^{3/2} behaviour at the break points."""
    d = np.atleast_1d(np.asarray(d, float))
    Rp = np.atleast_1d(np.asarray(Rp, float))
    d, Rp = np.broadcast_arrays(d, Rp)
    half = 0.5 * math.pi
    tb = []
    for rb in (np.abs(Rp - d), Rp + d):
        t = np.where((rb > 0) & (rb < sigma), np.arccos(np.clip(rb / sigma, -1, 1)), 0.0)
        tb.append(t)
    t1 = np.minimum(tb[0], tb[1])
    t2 = np.maximum(tb[0], tb[1])
    edges = [np.zeros_like(d), t1, t2, np.full_like(d, half)]
    u, wu = _gauss_legendre01(n_gl)
    total = np.zeros(d.shape)
    for a, b in zip(edges[:-1], edges[1:]):
        L = b - a
        m = L > 0
        if not np.any(m):
            continue
        aa, LL, dd, RR = a[m][:, None], L[m][:, None], d[m][:, None], Rp[m][:, None]
        phi = 0.5 * (1.0 - np.cos(math.pi * u))
        jac = 0.5 * math.pi * np.sin(math.pi * u)
        t = aa + LL * phi
        r = sigma * np.cos(t)
        integrand = circle_lens_area(r, dd, RR) * sigma * np.cos(t)
        total[m] += 2.0 * (integrand * (LL * jac * wu)).sum(axis=1)
    return total


def fm_weights(grid: Grid, sigma: float, n_gl: int = 64) -> np.ndarray:
    """Dense W (N x N): nbar_i = sum_j W_ij n_j  (Eq. fm with n = 0 outside the domain)."""
    N = grid.N
    W = np.zeros((N, N))
    norm = 3.0 / (4.0 * math.pi * sigma ** 3)
    full = 4.0 / 3.0 * math.pi * sigma ** 3
    for i in range(N):
        d = grid.R_c[i]
        Rp = grid.R_f
        U = np.zeros(N + 1)
        inside = d + sigma <= Rp
        U[inside] = full
        part = (~inside) & (Rp > d - sigma) & (Rp > 0)
        if grid.geometry == SPH:
            U[part] = lens_volume(sigma, Rp[part], d)
        else:
            U[part] = ball_cylinder_volume(sigma, d, Rp[part], n_gl)
        W[i] = norm * (U[1:] - U[:-1])
    return W
