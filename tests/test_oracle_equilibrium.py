"""Pins of the oracle's discrete equilibria (Sec. III.C): Gaussian moments, the T = 1, u = 0
limit, and the paper's printed half-range form (Eq. eq_gak_hh) written out independently here."""
import math

import numpy as np
import pytest
from numpy.polynomial import polynomial as Pnp
from scipy.integrate import quad as integrate
from scipy.special import comb, erf

from oracle import equilibrium as eq
from oracle import quadrature as quad

CASES = [(0.0, 1.0), (0.1, 1.0), (-0.3, 1.2), (0.25, 0.8), (0.05, 1.3)]


def gaussian_moment(m, u, T):
    """E[X^m] for X ~ N(u, T)."""
    tot = 0.0
    for j in range(0, m + 1, 2):
        dfact = float(np.prod(np.arange(j - 1, 0, -2))) if j else 1.0
        tot += comb(m, j) * u ** (m - j) * T ** (j / 2) * dfact
    return tot


@pytest.mark.parametrize("Q,N", [(4, 3), (8, 7), (12, 7)])
@pytest.mark.parametrize("u,T", CASES)
def test_full_range_moments_are_gaussian(Q, N, u, T):
    p, w = quad.full_range_rule(Q)
    g = eq.g_full(p, w, N, u, T)
    for m in range(N + 1):
        assert (g * p ** m).sum() == pytest.approx(gaussian_moment(m, u, T), rel=1e-12, abs=1e-13)


@pytest.mark.parametrize("Q", [2, 4, 8, 12])
def test_equilibrium_at_reference_state_is_the_weights(Q):
    p, w = quad.full_range_rule(Q)
    assert np.allclose(eq.g_full(p, w, Q - 1, 0.0, 1.0), w, rtol=1e-13, atol=1e-15 * w.max())
    x, lam, a, b = quad.half_range_rule(Q)
    ph, wh = np.concatenate([x, -x]), np.concatenate([lam, lam])
    assert np.allclose(eq.g_half(ph, wh, a, b, min(Q - 1, 7), 0.0, 1.0), wh, rtol=1e-12, atol=1e-15 * wh.max())


@pytest.mark.parametrize("Q,N", [(4, 3), (8, 7), (12, 7)])
@pytest.mark.parametrize("u,T", CASES)
def test_half_range_half_line_moments(Q, N, u, T):
    # on each half line the discrete g reproduces int_0^inf x^m G(+-x) dx for m <= N
    x, lam, a, b = quad.half_range_rule(Q)
    ph, wh = np.concatenate([x, -x]), np.concatenate([lam, lam])
    g = eq.g_half(ph, wh, a, b, N, u, T)
    G = lambda y: math.exp(-(y - u) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)
    for m in range(N + 1):
        plus = integrate(lambda y: y ** m * G(y), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        minus = integrate(lambda y: y ** m * G(-y), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        assert (g[:Q] * x ** m).sum() == pytest.approx(plus, rel=1e-10, abs=1e-13)
        assert (g[Q:] * x ** m).sum() == pytest.approx(minus, rel=1e-10, abs=1e-13)


def _P_plus_minus(S):
    """P_s^+(x) = e^{-x^2} d^s/dx^s e^{x^2},  P_s^-(x) = e^{x^2} d^s/dx^s e^{-x^2}
    as coefficient arrays (Sec. III.C)."""
    Pp, Pm = [np.array([1.0])], [np.array([1.0])]
    for _ in range(S):
        Pp.append(Pnp.polyadd(Pnp.polymulx(2 * Pp[-1]), Pnp.polyder(Pp[-1])))
        Pm.append(Pnp.polyadd(Pnp.polymulx(-2 * Pm[-1]), Pnp.polyder(Pm[-1])))
    return Pp, Pm


def printed_half_range_equilibrium(Q, N, u, T):
    """g^h_k = (w_k/2) sum_{s<=N} (T/2)^{s/2} Phi_s^N(|p_k|) [(1 + erf z) P_s^+(z)
    + (2/sqrt(pi)) e^{-z^2} P_s^*(z)],  z = +-u/sqrt(2T) by the sign of p_k,
    Phi_s^N(x) = sum_{l=s}^N h_{l,s} h_l(x),  P_s^* = sum_{j<s} C(s,j) P_j^+ P_{s-j-1}^-
    (Eq. eq_gak_hh, as printed)."""
    x, lam, a, b = quad.half_range_rule(Q)
    C = quad.half_poly_coeffs(a, b, N)
    H = quad.half_poly(x, a, b, N)
    Pp, Pm = _P_plus_minus(N)
    out = []
    for sgn in (+1.0, -1.0):
        z = sgn * u / math.sqrt(2 * T)
        g = np.zeros(Q)
        for s in range(N + 1):
            Phi = sum(C[l, s] * H[l] for l in range(s, N + 1))
            Pstar = sum(comb(s, j) * Pnp.polyval(z, Pp[j]) * Pnp.polyval(z, Pm[s - j - 1]) for j in range(s))
            bracket = (1 + erf(z)) * Pnp.polyval(z, Pp[s]) + 2 / math.sqrt(math.pi) * math.exp(-z * z) * Pstar
            g += (T / 2) ** (s / 2) * Phi * bracket
        out.append(0.5 * lam * g)
    return np.concatenate(out)


@pytest.mark.parametrize("Q,N", [(2, 1), (4, 3), (8, 7), (12, 7)])
@pytest.mark.parametrize("u,T", CASES)
def test_half_range_equals_printed_formula(Q, N, u, T):
    x, lam, a, b = quad.half_range_rule(Q)
    ph, wh = np.concatenate([x, -x]), np.concatenate([lam, lam])
    ours = eq.g_half(ph, wh, a, b, N, u, T)
    printed = printed_half_range_equilibrium(Q, N, u, T)
    assert np.allclose(ours, printed, rtol=1e-9, atol=1e-14 * np.max(np.abs(printed)))


def test_half_range_mass_is_one():
    x, lam, a, b = quad.half_range_rule(8)
    ph, wh = np.concatenate([x, -x]), np.concatenate([lam, lam])
    for u, T in CASES:
        assert eq.g_half(ph, wh, a, b, 7, u, T).sum() == pytest.approx(1.0, rel=1e-13)
