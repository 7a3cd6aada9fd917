"""Gauss-Hermite quadrature rules of the mixed-quadrature model (paper Sec. III.A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Both rules integrate against the normal weight omega(x) = exp(-x^2/2)/sqrt(2 pi)
(Sec. III.A, definition of omega below the population formula):

* full range  (HLB):  nodes are the roots of the probabilists' Hermite polynomial He_Q,
  weights sum to 1;
* half range  (HHLB): on each half line [0, inf) the nodes are the roots of the
  polynomial h_Q orthonormal under omega restricted to [0, inf); the negative nodes
  mirror the positive ones.  Indices 0..Q-1 hold the positive nodes, Q..2Q-1 the
  negative ones, in the same order (Sec. III.A, index convention).  Each half carries
  weight 1/2.

Construction (plain definitions):

* full range: the Jacobi matrix of the three-term recurrence He_{n+1} = x He_n - n He_{n-1}
  (Golub-Welsch), eigen-decomposed with numpy.
* half range: exact half-line moments mu_k = int_0^inf x^k omega(x) dx, turned into
  recurrence coefficients by the Chebyshev algorithm carried out in 60+ digit decimal
  arithmetic, then Golub-Welsch in FP64.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext, localcontext

import numpy as np


# ----------------------------------------------------------------------------- full range
def full_range_rule(Q: int):
    """Nodes (ascending) and weights of the Q-point full-range Gauss-Hermite rule.

    Sec. III.A: nodes are the roots of He_Q; the weight function is omega, so the weights
    sum to 1.  Golub-Welsch on the recurrence He_{n+1} = x He_n - n He_{n-1}.
    """
    if Q < 1:
        raise ValueError("Q >= 1")
    J = np.zeros((Q, Q))
    for n in range(1, Q):
        J[n, n - 1] = J[n - 1, n] = math.sqrt(n)
    x, V = np.linalg.eigh(J)
    w = V[0, :] ** 2  # total mass of omega is 1
    order = np.argsort(x)
    return x[order].copy(), w[order].copy()


def hermite_he(x, L: int):
    """He_0(x) .. He_L(x) (probabilists' Hermite), stacked on a new leading axis."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((L + 1,) + x.shape)
    out[0] = 1.0
    if L >= 1:
        out[1] = x
    for n in range(1, L):
        out[n + 1] = x * out[n] - n * out[n - 1]
    return out


# ----------------------------------------------------------------------------- half range
def _dec_pi(prec: int) -> Decimal:
    """pi to `prec` digits by Machin's formula pi = 16 atan(1/5) - 4 atan(1/239)."""
    with localcontext() as ctx:
        ctx.prec = prec + 10

        def atan_inv(n: int) -> Decimal:
            x = Decimal(1) / n
            x2 = x * x
            term = x
            total = x
            k = 1
            eps = Decimal(10) ** (-(prec + 8))
            while abs(term) > eps:
                term *= -x2
                total += term / (2 * k + 1)
                k += 1
            return total

        return +(16 * atan_inv(5) - 4 * atan_inv(239))


def half_line_moments_exact(K: int, prec: int):
    """mu_k = int_0^inf x^k omega(x) dx for k = 0..K-1 as Decimals.

    mu_{2m} = (2m-1)!!/2 and mu_{2m+1} = 2^m m!/sqrt(2 pi)  (Gaussian integrals).
    """
    with localcontext() as ctx:
        ctx.prec = prec
        s2pi = (2 * _dec_pi(prec)).sqrt()
        mu = []
        for k in range(K):
            if k % 2 == 0:
                m = k // 2
                dfact = 1
                for j in range(1, 2 * m, 2):
                    dfact *= j
                mu.append(Decimal(dfact) / 2)
            else:
                m = (k - 1) // 2
                mu.append(Decimal(2 ** m * math.factorial(m)) / s2pi)
        return mu


def half_range_recurrence(Q: int, prec: int | None = None):
    """Recurrence coefficients (alpha_k, beta_k), k = 0..Q-1, of the monic polynomials
    orthogonal under omega on [0, inf).  beta_0 = mu_0 = 1/2 (the mass of one half line).

    Chebyshev's algorithm (moments -> recurrence) in high-precision decimal arithmetic,
    because the map is ill-conditioned in FP64.
    """
    if prec is None:
        prec = 60 + 4 * Q
    mu = half_line_moments_exact(2 * Q, prec)
    with localcontext() as ctx:
        ctx.prec = prec
        n = Q
        alpha = [Decimal(0)] * n
        beta = [Decimal(0)] * n
        sig_prev = [Decimal(0)] * (2 * n)  # sigma_{-1, l}
        sig = list(mu)  # sigma_{0, l}
        alpha[0] = mu[1] / mu[0]
        beta[0] = mu[0]
        for k in range(1, n):
            sig_new = [Decimal(0)] * (2 * n)
            for l in range(k, 2 * n - k):
                sig_new[l] = sig[l + 1] - alpha[k - 1] * sig[l] - beta[k - 1] * sig_prev[l]
            alpha[k] = sig_new[k + 1] / sig_new[k] - sig[k] / sig[k - 1]
            beta[k] = sig_new[k] / sig[k - 1]
            sig_prev, sig = sig, sig_new
        return np.array([float(a) for a in alpha]), np.array([float(b) for b in beta])


def half_range_rule(Q: int):
    """Positive nodes (ascending) x_1..x_Q and weights lambda (summing to 1/2) of the
    Q-point half-range rule, plus the recurrence coefficients used to build them.

    Nodes: the eigenvalues of the Jacobi matrix (the roots of h_Q).  Weights: the closed form of
    Sec. III.A, w_i = x_i a_{Q-1}^2 / (h_{Q-1}(x_i)^2 [x_i + h_Q(0)^2 / sqrt(2 pi)]) with
    a_{Q-1} = (leading coefficient of h_Q) / (that of h_{Q-1}) = 1 / sqrt(beta_Q); it keeps its
    relative accuracy for the smallest weights (below 1e-100 at Q = 100), which the first
    components of the Jacobi matrix's eigenvectors do not.
    """
    alpha, beta = half_range_recurrence(Q + 1)
    J = np.diag(alpha[:Q])
    for k in range(1, Q):
        J[k, k - 1] = J[k - 1, k] = math.sqrt(beta[k])
    x = np.sort(np.linalg.eigvalsh(J))
    H = half_poly(np.concatenate([x, [0.0]]), alpha, beta, Q)
    hQ0 = H[Q, -1]
    a = 1.0 / math.sqrt(beta[Q])
    lam = x * a ** 2 / (H[Q - 1, :Q] ** 2 * (x + hQ0 ** 2 / math.sqrt(2.0 * math.pi)))
    return x, lam, alpha[:Q].copy(), beta[:Q].copy()


def half_range_axis(Q: int):
    """The 2Q nodes and weights of a half-range axis in the paper's index order:
    positive nodes first (ascending), then their mirror images (Sec. III.A)."""
    x, lam, _, _ = half_range_rule(Q)
    return np.concatenate([x, -x]), np.concatenate([lam, lam])


def half_poly(x, alpha, beta, L: int):
    """h_0(x)..h_L(x), the polynomials orthonormal under omega on [0, inf)
    (int_0^inf omega h_l h_m = delta_lm, so h_0 = sqrt(2)), by the three-term recurrence
    b_{l+1} h_{l+1} = (x - alpha_l) h_l - b_l h_{l-1},  b_l = sqrt(beta_l)."""
    x = np.asarray(x, dtype=np.float64)
    b = np.sqrt(beta)
    out = np.empty((L + 1,) + x.shape)
    out[0] = 1.0 / b[0]
    if L >= 1:
        out[1] = (x - alpha[0]) * out[0] / b[1]
    for l in range(1, L):
        out[l + 1] = ((x - alpha[l]) * out[l] - b[l] * out[l - 1]) / b[l + 1]
    return out


def half_poly_coeffs(alpha, beta, L: int):
    """Monomial coefficients C[l, s] of h_l(x) = sum_s C[l, s] x^s (the h_{l,s} of Sec. III.A)."""
    b = np.sqrt(beta)
    C = np.zeros((L + 1, L + 1))
    C[0, 0] = 1.0 / b[0]
    if L >= 1:
        C[1, 1] = C[0, 0] / b[1]
        C[1, 0] = -alpha[0] * C[0, 0] / b[1]
    for l in range(1, L):
        xh = np.zeros(L + 1)
        xh[1:] = C[l, :-1]
        C[l + 1] = (xh - alpha[l] * C[l] - b[l] * C[l - 1]) / b[l + 1]
    return C


def half_poly_deriv(x, alpha, beta, L: int):
    """h_0'(x)..h_L'(x) by differentiating the three-term recurrence:
    b_{l+1} h'_{l+1} = h_l + (x - alpha_l) h'_l - b_l h'_{l-1}."""
    x = np.asarray(x, dtype=np.float64)
    b = np.sqrt(beta)
    H = half_poly(x, alpha, beta, L)
    out = np.zeros((L + 1,) + x.shape)
    if L >= 1:
        out[1] = H[0] / b[1]
    for l in range(1, L):
        out[l + 1] = (H[l] + (x - alpha[l]) * out[l] - b[l] * out[l - 1]) / b[l + 1]
    return out
