"""Pins of the oracle's grid and Fischer-Methfessel weights (Sec. IV domain, Eq. fm, App. A)."""
import math

import numpy as np
import pytest
from scipy.special import elliprd, elliprf, elliprj

from oracle import geometry as geo


def _mc_volume(sigma, inside, n=2_000_000, seed=0):
    """Monte Carlo volume of {x in ball(sigma, 0)} for which inside(x) holds."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(-sigma, sigma, (n, 3))
    P = P[(P ** 2).sum(1) < sigma * sigma]
    frac = inside(P).mean()
    return frac * 4.0 / 3.0 * math.pi * sigma ** 3, 4.0 / 3.0 * math.pi * sigma ** 3 / math.sqrt(len(P))


@pytest.mark.parametrize("r2,d", [(1.0, 1.1), (1.0, 0.9), (0.5, 0.3), (2.0, 2.25), (0.1, 0.15)])
def test_lens_volume_against_monte_carlo(r2, d):
    sigma = 0.3
    ref, err = _mc_volume(sigma, lambda P: np.sqrt((P[:, 0] + d) ** 2 + P[:, 1] ** 2 + P[:, 2] ** 2) < r2)
    assert geo.lens_volume(sigma, r2, d)[()] == pytest.approx(ref, abs=5 * err)


def test_lens_volume_special_cases():
    s = 0.4
    assert geo.lens_volume(s, 2.0, 1.0)[()] == pytest.approx(4 / 3 * math.pi * s ** 3)  # nested
    assert geo.lens_volume(s, 1.0, 1.5)[()] == 0.0  # disjoint
    # equal spheres at distance d: pi (4 r + d)(2 r - d)^2 / 12
    r, d = 0.5, 0.3
    assert geo.lens_volume(r, r, d)[()] == pytest.approx(math.pi * (4 * r + d) * (2 * r - d) ** 2 / 12, rel=1e-14)


def _ellK(k):
    """Complete elliptic integral of the first kind in Carlson's form, K = R_F(0, 1 - k^2, 1)."""
    return float(elliprf(0.0, 1.0 - k * k, 1.0))


def _ellE(k):
    """Second kind: E = R_F(0, 1 - k^2, 1) - (k^2 / 3) R_D(0, 1 - k^2, 1)."""
    m = k * k
    return float(elliprf(0.0, 1.0 - m, 1.0) - m / 3.0 * elliprd(0.0, 1.0 - m, 1.0))


def _ellPi(k, a2):
    """Third kind, int_0^{pi/2} dt / ((1 - a2 sin^2 t) sqrt(1 - k^2 sin^2 t))
    = R_F(0, 1 - k^2, 1) + (a2 / 3) R_J(0, 1 - k^2, 1, 1 - a2)."""
    m = k * k
    return float(elliprf(0.0, 1.0 - m, 1.0) + a2 / 3.0 * elliprj(0.0, 1.0 - m, 1.0, 1.0 - a2))


def paper_sphere_cylinder_volume(r, R, b):
    """App. A (Lamarche-Leroy) sphere(radius r, centre at distance b from the axis) cap
    cylinder(radius R), for r < R and r < b + R.  Readings: E(k) is the standard complete
    integral of the second kind (the printed integrand swaps sqrt(1-z^2) and sqrt(1-k^2 z^2));
    Pi uses the printed integrand 1/(1 - alpha^2 z^2) with -alpha^2 = (B - C)/C."""
    A = max(r * r, (b + R) ** 2)
    B = min(r * r, (b + R) ** 2)
    C = (b - R) ** 2
    k = math.sqrt((B - C) / (A - C))
    alpha2 = -(B - C) / C
    s = (b + R) * (b - R)
    theta = 1.0 if R - b > 0 else 0.0
    return 4 * math.pi / 3 * r ** 3 * theta + 4 / (3 * math.sqrt(A - C)) * (
        _ellPi(k, alpha2) * B * B * s / C
        + _ellK(k) * (s * (A - 2 * B) + (A - B) * (3 * B - C - 2 * A) / 3)
        + _ellE(k) * (A - C) * (-s + (2 * A + 2 * C - 4 * B) / 3))


@pytest.mark.parametrize("r,R,b", [(0.3, 1.0, 1.1), (0.3, 1.0, 0.9), (0.3, 1.0, 1.25), (0.2, 1.2, 1.3),
                                   (0.45, 2.0, 1.7), (0.11, 1.5, 1.45)])
def test_ball_cylinder_volume_matches_appendix_A_formula(r, R, b):
    ours = geo.ball_cylinder_volume(r, b, R)[0]
    assert ours == pytest.approx(paper_sphere_cylinder_volume(r, R, b), rel=1e-11)


def test_ball_cylinder_volume_on_axis_closed_form():
    # ball centred on the axis: (4 pi / 3)(s^3 - (s^2 - R^2)^{3/2}) for R < s
    s = 0.5
    for R in (0.1, 0.3, 0.49):
        exact = 4 * math.pi / 3 * (s ** 3 - (s * s - R * R) ** 1.5)
        assert geo.ball_cylinder_volume(s, 0.0, R)[0] == pytest.approx(exact, rel=1e-12)


def test_ball_cylinder_volume_against_monte_carlo_when_ball_wider_than_cylinder():
    sigma, d, R = 0.6, 0.5, 0.4
    ref, err = _mc_volume(sigma, lambda P: np.hypot(P[:, 0] + d, P[:, 1]) < R)
    assert geo.ball_cylinder_volume(sigma, d, R)[0] == pytest.approx(ref, abs=5 * err)


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_fm_weights_rows_sum_to_one_away_from_walls(g, beta):
    sigma = 0.25
    G = geo.make_grid(g, 1.0, 3.0, sigma, 96, beta)
    W = geo.fm_weights(G, sigma)
    lo, hi = G.R_f[0], G.R_f[-1]
    inner = (G.R_c - sigma >= lo) & (G.R_c + sigma <= hi)
    assert inner.sum() > 10
    assert np.allclose(W[inner].sum(1), 1.0, rtol=1e-12)
    # near the walls part of the ball lies outside the fluid: n = 0 there (A4 reading)
    assert W[0].sum() < 0.75 and W[-1].sum() < 0.75
    assert np.all(W >= -1e-15)


@pytest.mark.parametrize("g", [geo.CYL, geo.SPH])
def test_grid_volumes_and_curvature(g):
    sigma = 0.2
    G = geo.make_grid(g, 1.0, 2.0, sigma, 50, 1.5)
    a, b = 1.0 + sigma / 2, 2.0 - sigma / 2
    total = (b * b - a * a) / 2 if g == geo.CYL else (b ** 3 - a ** 3) / 3
    assert G.V_c.sum() == pytest.approx(total, rel=1e-14)
    assert G.R_f[0] == pytest.approx(a) and G.R_f[-1] == pytest.approx(b)
    Rm = 0.5 * (G.R_f[1:] + G.R_f[:-1])
    if g == geo.CYL:
        assert np.allclose(G.kappa, 1.0 / Rm, rtol=1e-13)
    else:
        # (r+^2 - r-^2) / ((r+^3 - r-^3)/3) -> 2/r as the cells shrink
        assert np.allclose(G.kappa, 2.0 / Rm, rtol=1e-3)
    assert np.all(np.diff(G.R_c) > 0)
