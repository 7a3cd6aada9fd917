"""Pins of the oracle's momentum-derivative matrices (Sec. III.B): exact derivatives of
Hermite-Gaussian functions, moment identities, and the paper's printed half-range form."""
import math

import numpy as np
import pytest

from oracle import kmatrix as km
from oracle import quadrature as quad


@pytest.mark.parametrize("Q", [2, 4, 8, 12])
def test_k1_full_differentiates_hermite_gaussians(Q):
    # f = omega He_m  ->  d f/dp = -omega He_{m+1}; weighted: K1 (w He_m) = -w He_{m+1}, m <= Q-1
    p, w = quad.full_range_rule(Q)
    He = quad.hermite_he(p, Q + 1)
    K = km.k1_full(p, w)
    for m in range(Q):
        scale = np.max(np.abs(w * He[m + 1])) + 1e-300
        assert np.allclose(K @ (w * He[m]), -w * He[m + 1], atol=1e-11 * max(scale, 1.0))


@pytest.mark.parametrize("Q", [2, 3, 4, 8, 12])
def test_k2_full_differentiates_p_times_hermite_gaussians(Q):
    # d(p omega He_m)/dp = -omega (He_{m+2} + m He_m), m <= Q-2
    p, w = quad.full_range_rule(Q)
    He = quad.hermite_he(p, Q + 2)
    K = km.k2_full(p, w)
    for m in range(Q - 1):
        exact = -w * (He[m + 2] + m * He[m])
        assert np.allclose(K @ (w * He[m]), exact, atol=1e-11 * max(np.max(np.abs(exact)), 1.0))


def _half(Q):
    x, lam, a, b = quad.half_range_rule(Q)
    return np.concatenate([x, -x]), np.concatenate([lam, lam]), a, b


@pytest.mark.parametrize("Q", [4, 6, 8, 12])
def test_k_half_exact_on_smooth_polynomial_gaussians(Q):
    # f(p) = omega(p)(1 + a p + b p^2): continuous at 0, so no jump; the derivative
    # omega(p)[a + 2 b p - p (1 + a p + b p^2)] is a cubic per half line: exact for Q >= 4.
    p, w, al, be = _half(Q)
    K = km.k1_half(p, w, al, be)
    A, B = 0.3, -0.2
    f = w * (1 + A * p + B * p * p)
    exact = w * (A + 2 * B * p - p * (1 + A * p + B * p * p))
    assert np.allclose(K @ f, exact, atol=1e-11 * np.max(np.abs(exact)))


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 12])
def test_k_half_moment_identities(Q):
    # int dp df/dp = 0, int p df/dp = -int f, int p^2 df/dp = -2 int p f (Q >= 3)
    p, w, al, be = _half(Q)
    K = km.k1_half(p, w, al, be)
    # K acts on weighted populations f_i' ~ w_i': compare the identities column by column
    # scaled by w_i' (the entries of K grow like 1/w_i' at the outer nodes)
    assert np.allclose(K.sum(0) * w, 0.0, atol=1e-13)
    if Q >= 2:
        assert np.allclose((p @ K) * w, -w, atol=1e-13)
    if Q >= 3:
        assert np.allclose(((p * p) @ K) * w, -2 * p * w, atol=1e-13)


def printed_k_half(Q):
    """K^h_{ii'} = w_i s_i { (1 + s_i s_i')/2 sum_{l=0}^{Q-2} h_l(|p_i'|) [ h_{l,0}/sqrt(2 pi)
    sum_{s=l+1}^{Q-1} h_{s,0} h_s(|p_i|) - (h_{l,l}/h_{l+1,l+1}) h_{l+1}(|p_i|) ]
    - Phi_0(|p_i|) Phi_0(|p_i'|) / (2 sqrt(2 pi)) }  (Sec. III.B, Eq. force1, half range,
    with the radial-axis labels of the last term read as the same axis; Phi_0 summed to Q-1)."""
    p, w, al, be = _half(Q)
    x, s = np.abs(p), np.sign(p)
    a2, b2 = quad.half_range_recurrence(Q + 1)
    C = quad.half_poly_coeffs(a2, b2, Q)
    H = quad.half_poly(x, a2, b2, Q)
    h0 = C[:, 0]
    Phi0 = sum(h0[l] * H[l] for l in range(Q))
    n = 2 * Q
    K = np.zeros((n, n))
    r2p = math.sqrt(2 * math.pi)
    for i in range(n):
        for j in range(n):
            acc = 0.0
            if s[i] == s[j]:
                for l in range(Q - 1):
                    inner = h0[l] / r2p * sum(h0[t] * H[t, i] for t in range(l + 1, Q))
                    inner -= C[l, l] / C[l + 1, l + 1] * H[l + 1, i]
                    acc += H[l, j] * inner
            acc -= Phi0[i] * Phi0[j] / (2 * r2p)
            K[i, j] = w[i] * s[i] * acc
    return K


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 12])
def test_k_half_equals_printed_form(Q):
    p, w, al, be = _half(Q)
    ours = km.k1_half(p, w, al, be)
    printed = printed_k_half(Q)
    assert np.allclose(ours, printed, atol=1e-11 * np.max(np.abs(printed)))
