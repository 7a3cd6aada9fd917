"""Momentum-derivative matrices of the force terms (paper Sec. III.B, Eqs. force1, force2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

All matrices act on weighted populations f_i = w_i f(p_i) / omega(p_i) along one axis:
(d f / d p)_i = sum_i' K1_{ii'} f_i'  and  (d (f p) / d p)_i = sum_i' K2_{ii'} f_i'.

* Full range: K1^H and K2^H as printed in Sec. III.B.
* Half range, d/dp (the radial axis): the plain definition.  On each half line f is
  represented as omega(p) sum_{l<Q} c_l^s h_l(|p|); d/dp is taken in the sense of
  distributions, so the jump f(0+) - f(0-) contributes a delta at p = 0, which is split
  equally between the two halves; the result is projected back on the same basis.  This
  gives
      K^h_{ii'} = -s_i w_i [ Phi0(|p_i|) Phi0(|p_i'|) / (2 sqrt(2 pi))
                             + delta_{s_i s_i'} sum_{l<Q} h_l(|p_i|) h_l'(|p_i'|) ],
  Phi0(x) = sum_{l<Q} h_l(0) h_l(x), which integration by parts turns into the printed
  form of Sec. III.B (checked in the tests).
"""
from __future__ import annotations

import math

import numpy as np

from .quadrature import half_poly, half_poly_deriv, hermite_he


def k1_full(p, w):
    """K^{H}_{ii'} = -w_i sum_{l=0}^{Q-1} He_{l+1}(p_i) He_l(p_i') / l!   (Eq. force1, full range)."""
    Q = len(p)
    He = hermite_he(p, Q)
    K = np.zeros((Q, Q))
    for l in range(Q):
        K -= np.outer(w * He[l + 1], He[l]) / math.factorial(l)
    return K


def k2_full(p, w):
    """K^{H}_{ii'} = -w_i sum_{l=0}^{Q-2} He_{l+1}(p_i) [He_{l+1}(p_i') + l He_{l-1}(p_i')] / l!
    (Eq. force2, full range)."""
    Q = len(p)
    He = hermite_he(p, Q)
    K = np.zeros((Q, Q))
    for l in range(Q - 1):
        right = He[l + 1] + (l * He[l - 1] if l >= 1 else 0.0)
        K -= np.outer(w * He[l + 1], right) / math.factorial(l)
    return K


def k1_half(p, w, alpha, beta):
    """Half-range d/dp matrix from the plain definition (module docstring).

    p, w: the 2Q nodes/weights in the paper's order; alpha, beta: recurrence coefficients.
    """
    n2 = len(p)
    Q = n2 // 2
    x = np.abs(p)
    s = np.sign(p)
    H = half_poly(x, alpha, beta, Q - 1)  # (Q, 2Q)
    dH = half_poly_deriv(x, alpha, beta, Q - 1)  # (Q, 2Q)
    h0 = half_poly(np.zeros(1), alpha, beta, Q - 1)[:, 0]  # h_l(0)
    Phi0 = h0 @ H  # (2Q,)
    same = (s[:, None] == s[None, :]).astype(np.float64)
    jump = np.outer(Phi0, Phi0) / (2.0 * math.sqrt(2.0 * math.pi))
    proj = H.T @ dH  # [i, i'] = sum_l h_l(x_i) h_l'(x_i')
    return -(s * w)[:, None] * (jump + same * proj)
