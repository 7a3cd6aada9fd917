"""Discrete per-axis equilibria of the factorised Maxwellian (paper Sec. III.C).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

f^MB_{ijk} = n g_{R,i} g_{2,j} g_{3,k}; each g is the weighted population of a 1-D Gaussian
N(u, T) expanded to order N on one quadrature axis:

* full range (Eq. eq_gak_H): g_k = w_k sum_{l<=N} He_l(p_k) sum_s (T-1)^s u^{l-2s} / (2^s s! (l-2s)!);
* half range: on the half line of sign s_k, the Gaussian restricted to it is projected on
  the orthonormal h_0..h_N, g_k = w_k sum_{l<=N} h_l(|p_k|) M_l^{s_k} with
  M_l^s = int_0^inf h_l(x) G(s x) dx.  This is the plain definition behind Eq. eq_gak_hh;
  M_l^s is formed from the half-line moments m_j of N(s u, T) on [0, inf):
  m_0 = (1 + erf(v / sqrt(2T))) / 2,  m_1 = v m_0 + T G_v(0),  m_{j+1} = v m_j + j T m_{j-1}.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .quadrature import half_poly, half_poly_coeffs, hermite_he


def g_full(p, w, N: int, u, T):
    """Full-range equilibrium vector (Eq. eq_gak_H), literally.

    p, w: nodes and weights (Q,).  u, T: arrays of any common shape S.  Returns S + (Q,).
    """
    u = np.asarray(u, dtype=np.float64)[..., None]
    T = np.asarray(T, dtype=np.float64)[..., None]
    He = hermite_he(p, N)  # (N+1, Q)
    out = np.zeros(np.broadcast(u, T).shape[:-1] + (len(p),))
    for l in range(N + 1):
        coef = 0.0
        for s in range(l // 2 + 1):
            coef = coef + (T - 1.0) ** s * u ** (l - 2 * s) / (
                2.0 ** s * math.factorial(s) * math.factorial(l - 2 * s))
        out = out + He[l] * coef
    return out * w


def half_line_gauss_moments(v, T, J: int):
    """m_j = int_0^inf x^j G_v(x) dx, j = 0..J, for G_v the N(v, T) density."""
    v = np.asarray(v, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    m = np.empty((J + 1,) + np.broadcast(v, T).shape)
    m[0] = 0.5 * (1.0 + erf(v / np.sqrt(2.0 * T)))
    G0 = np.exp(-v * v / (2.0 * T)) / np.sqrt(2.0 * math.pi * T)
    if J >= 1:
        m[1] = v * m[0] + T * G0
    for j in range(1, J):
        m[j + 1] = v * m[j] + j * T * m[j - 1]
    return m


def g_half(p, w, alpha, beta, N: int, u, T):
    """Half-range equilibrium vector (plain definition of Eq. eq_gak_hh).

    p, w: the 2Q nodes/weights in the paper's order (positive half first).
    alpha, beta: half-range recurrence coefficients.  Returns shape S + (2Q,).
    """
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    C = half_poly_coeffs(alpha, beta, N)  # (N+1, N+1)
    H = half_poly(np.abs(p), alpha, beta, N)  # (N+1, 2Q)
    sign = np.sign(p)
    out = np.zeros(np.broadcast(u, T).shape + (len(p),))
    for half in (+1.0, -1.0):
        m = half_line_gauss_moments(half * u, T, N)  # (N+1,) + S
        M = np.tensordot(C, m, axes=([1], [0]))  # (N+1,) + S : M_l
        sel = sign == half
        val = np.tensordot(np.moveaxis(M, 0, -1), H[:, sel], axes=([-1], [0]))
        out[..., sel] = val
    return out * w
