"""Pins of the oracle's quadrature rules (Sec. III.A) against closed forms, a library
routine and the weight formulas printed in the paper."""
import math

import numpy as np
import pytest
from scipy.special import gamma

from oracle import quadrature as quad


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 12, 16])
def test_full_range_matches_numpy_hermegauss(Q):
    x, w = quad.full_range_rule(Q)
    xr, wr = np.polynomial.hermite_e.hermegauss(Q)
    assert np.allclose(x, xr, atol=1e-13)
    assert np.allclose(w, wr / math.sqrt(2 * math.pi), rtol=1e-11)


@pytest.mark.parametrize("Q", [1, 2, 4, 8, 12])
def test_full_range_exact_on_gaussian_moments(Q):
    # sum w p^k = E[X^k] for X ~ N(0, 1): (k-1)!! for even k, 0 for odd, for all k < 2Q
    x, w = quad.full_range_rule(Q)
    for k in range(2 * Q):
        exact = 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0
        scale = (w * np.abs(x) ** k).sum()  # rounding of the sum scales with its terms
        assert abs((w * x ** k).sum() - exact) <= 1e-13 * scale


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 12])
def test_full_range_weight_formula_of_the_paper(Q):
    # w_i^H = Q! / He_{Q+1}(p_i)^2  (Sec. III.A)
    x, w = quad.full_range_rule(Q)
    He = quad.hermite_he(x, Q + 1)
    assert np.allclose(w, math.factorial(Q) / He[Q + 1] ** 2, rtol=1e-11)


def _half_moment(k):
    return 2.0 ** ((k - 1) / 2.0) * gamma((k + 1) / 2.0) / math.sqrt(2 * math.pi)


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 12, 20, 32, 48, 64, 100])
def test_half_range_exact_on_half_line_moments(Q):
    # up to the orders of the paper's Couette runs (HHLB(7,20), HHLB(7,100), Sec. IV.A)
    x, lam, _, _ = quad.half_range_rule(Q)
    assert np.all(x > 0)
    for k in range(2 * Q):
        assert (lam * x ** k).sum() == pytest.approx(_half_moment(k), rel=2e-13 if Q <= 20 else 2e-12)


def test_half_range_Q1_closed_form():
    # one node: mean of the half-normal sqrt(2/pi), weight 1/2
    x, lam, _, _ = quad.half_range_rule(1)
    assert x[0] == pytest.approx(math.sqrt(2 / math.pi), rel=1e-15)
    assert lam[0] == pytest.approx(0.5, rel=1e-15)


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 6, 8, 12])
def test_half_range_weights_match_golub_welsch(Q):
    # the oracle's weights follow the closed form of Sec. III.A; Golub-Welsch gives them as
    # beta_0 times the squared first components of the Jacobi matrix's eigenvectors (numpy eigh)
    x, lam, alpha, beta = quad.half_range_rule(Q)
    J = np.diag(alpha)
    for k in range(1, Q):
        J[k, k - 1] = J[k - 1, k] = math.sqrt(beta[k])
    ev, V = np.linalg.eigh(J)
    order = np.argsort(ev)
    assert np.allclose(x, ev[order], rtol=1e-13)
    assert np.allclose(lam, beta[0] * V[0, order] ** 2, rtol=1e-10)


@pytest.mark.parametrize("Q", [2, 5, 12])
def test_half_polynomials_orthonormal_and_roots(Q):
    x, lam, alpha, beta = quad.half_range_rule(Q)
    H = quad.half_poly(x, alpha, beta, Q - 1)
    G = (H * lam) @ H.T
    assert np.allclose(G, np.eye(Q), atol=1e-12)
    assert quad.half_poly(np.zeros(1), alpha, beta, 0)[0, 0] == pytest.approx(math.sqrt(2))
    # the nodes are the roots of h_Q (needs alpha_Q, beta_Q: one more recurrence step)
    a2, b2 = quad.half_range_recurrence(Q + 1)
    Hx = quad.half_poly(x, a2, b2, Q)
    assert np.max(np.abs(Hx[Q]) / np.sqrt((Hx ** 2).sum(0))) < 1e-12


def test_half_range_axis_index_convention():
    # positive nodes first, then their mirror images (Sec. III.A)
    p, w = quad.half_range_axis(4)
    assert np.all(p[:4] > 0) and np.allclose(p[4:], -p[:4]) and np.allclose(w[4:], w[:4])
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
