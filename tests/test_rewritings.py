"""The exact rewritings the kernels use, restated in numpy and checked against the direct forms of
the formulas on random FP64 inputs (CPU): the ascending-window WENO5 for both upwind directions
(and its negation-free arrangement, evaluated on pairs of momenta),
the reconstruction of f itself with epsilon scaled by the squared weight,
the Shakhov factor and J1 as polynomials in x1 = p_2 - u_2 along a vector of momenta, and the
double-float split of an FP64 sum.  The kernels themselves are checked against the oracle by the
GPU tests; these pin the algebra the kernels were derived from."""
import numpy as np


def weno5_direct(a, b, c, d, e):
    eps = 1e-6
    t0, t1 = a - 2 * b + c, a - 4 * b + 3 * c
    t2, t3 = b - 2 * c + d, b - d
    t4, t5 = c - 2 * d + e, 3 * c - 4 * d + e
    be = [eps + 13 / 12 * t0 ** 2 + 0.25 * t1 ** 2, eps + 13 / 12 * t2 ** 2 + 0.25 * t3 ** 2,
          eps + 13 / 12 * t4 ** 2 + 0.25 * t5 ** 2]
    al = [0.1 / be[0] ** 2, 0.6 / be[1] ** 2, 0.3 / be[2] ** 2]
    r = [(2 * a - 7 * b + 11 * c) / 6, (-b + 5 * c + 2 * d) / 6, (2 * c + 5 * d - e) / 6]
    return sum(x * y for x, y in zip(al, r)) / sum(al)


def weno5_ascending(w0, w1, w2, w3, w4, sigma, e4=4e-6):
    d0, d1, d2, d3 = w1 - w0, w2 - w1, w3 - w2, w4 - w3
    D1, D2, D3 = d1 - d0, d2 - d1, d3 - d2
    tL, tC, tR = 3 * d1 - d0, -(d1 + d2), d3 - 3 * d2
    E = [tL ** 2 + 13 / 3 * D1 ** 2 + e4, tC ** 2 + 13 / 3 * D2 ** 2 + e4, tR ** 2 + 13 / 3 * D3 ** 2 + e4]
    m = np.minimum(E[0], np.minimum(E[1], E[2]))
    dL, dR = (0.1, 0.3) if sigma > 0 else (0.3, 0.1)
    a = [dL * (m / E[0]) ** 2, 0.6 * (m / E[1]) ** 2, dR * (m / E[2]) ** 2]
    s3 = 3.0 * sigma
    X = [D1 + s3 * tL, D2 - s3 * tC, D3 - s3 * tR]
    return w2 + sum(x * y for x, y in zip(a, X)) / (12 * sum(a))


def weno5_negation_free(w0, w1, w2, w3, w4, sigma, e4=4e-6):
    # the arrangement the stage kernel evaluates on pairs of momenta: -d0 and -tC enter instead of
    # d0 and tC, so that every step is one fused multiply-add, add or product
    nd0, d1, d2, d3 = w0 - w1, w2 - w1, w3 - w2, w4 - w3
    D1, D2, D3 = d1 + nd0, d2 - d1, d3 - d2
    tL, ntC, tR = 3 * d1 + nd0, d1 + d2, -3 * d2 + d3
    E = [tL * tL + (13 / 3 * D1) * D1 + e4, ntC * ntC + (13 / 3 * D2) * D2 + e4, tR * tR + (13 / 3 * D3) * D3 + e4]
    m = np.minimum(E[0], np.minimum(E[1], E[2]))
    dL, dR = (0.1, 0.3) if sigma > 0 else (0.3, 0.1)
    s = [m / E[0], m / E[1], m / E[2]]
    a = [dL * (s[0] * s[0]), 0.6 * (s[1] * s[1]), dR * (s[2] * s[2])]
    s3, ns3 = 3.0 * sigma, -3.0 * sigma
    X = [s3 * tL + D1, s3 * ntC + D2, ns3 * tR + D3]
    num = a[2] * X[2] + (a[1] * X[1] + a[0] * X[0])
    return w2 + num / (12 * ((a[0] + a[1]) + a[2]))


def test_ascending_weno5_equals_the_direct_form_both_directions():
    rng = np.random.default_rng(3)
    w = rng.normal(size=(5, 20000)) * np.exp(rng.normal(size=(5, 20000)))
    fwd = weno5_direct(*w)
    rev = weno5_direct(w[4], w[3], w[2], w[1], w[0])
    scale = np.max(np.abs(w), axis=0)
    assert np.max(np.abs(weno5_ascending(*w, +1) - fwd) / scale) < 1e-12
    assert np.max(np.abs(weno5_ascending(*w, -1) - rev) / scale) < 1e-12
    assert np.max(np.abs(weno5_negation_free(*w, +1) - fwd) / scale) < 1e-12
    assert np.max(np.abs(weno5_negation_free(*w, -1) - rev) / scale) < 1e-12


def test_weno5_of_f_with_scaled_epsilon_is_w_times_weno5_of_f_over_w():
    # the stage kernel reconstructs f = w g with 4 eps w^2; the method reconstructs g = f / w with
    # 4 eps: the face value of f is w times that of g (weights spanning the half-range rules' range)
    rng = np.random.default_rng(7)
    g = np.exp(rng.normal(size=(5, 20000))) * (1.0 + 0.3 * rng.normal(size=(5, 20000)))
    wt = 10.0 ** rng.uniform(-12, 0, size=20000)
    for sigma in (+1, -1):
        ref = wt * (weno5_direct(*g) if sigma > 0 else weno5_direct(g[4], g[3], g[2], g[1], g[0]))
        got = weno5_ascending(*(wt * g), sigma, e4=4e-6 * wt ** 2)
        assert np.max(np.abs(got - ref) / (wt * np.max(np.abs(g), axis=0))) < 1e-12


def test_collision_polynomials_equal_the_direct_form():
    rng = np.random.default_rng(5)
    n = 64
    pr, p2, p3 = rng.normal(size=(3, n))
    u0, u1, u2 = 0.2 * rng.normal(size=(3, n))
    iT, cS, brchi, X, Y, dv = rng.uniform(0.5, 2.0, size=(6, n))
    q0, q1, q2, S00, S11, S22, S01, S02 = 0.1 * rng.normal(size=(8, n))
    x0, x1, x2 = pr - u0, p2 - u1, p3 - u2
    # direct: Shakhov factor f^S / f^MB and J1 / f^MB
    xs, xq = x0 ** 2 + x1 ** 2 + x2 ** 2, x0 * q0 + x1 * q1 + x2 * q2
    z2 = 0.5 * xs * iT
    strain = iT * (x0 ** 2 * S00 + x1 ** 2 * S11 + x2 ** 2 * S22 + 2 * x0 * x1 * S01 + 2 * x0 * x2 * S02)
    j1 = -brchi * (x0 * (X + 0.6 * (z2 - 2.5) * Y) + 0.4 * (strain + (z2 - 2.5) * dv))
    shak = 1 + cS * (0.2 * xs * iT - 1) * xq
    # the kernel's coefficients (per vector: everything but x1)
    hiT, fiT = 0.5 * iT, 0.2 * iT
    xsA, xqA = x0 ** 2 + x2 ** 2, x0 * q0 + x2 * q2
    stA = x0 ** 2 * S00 + x2 ** 2 * S22 + 2 * x0 * x2 * S02
    Yd = 0.6 * x0 * Y + 0.4 * dv
    J0 = -brchi * (x0 * X + Yd * (hiT * xsA - 2.5) + 0.4 * iT * stA)
    J1 = -brchi * 0.4 * (2 * iT * S01) * x0
    J2 = -brchi * (Yd * hiT + 0.4 * iT * S11)
    b0 = fiT * xsA - 1
    F0, F1, F2, F3 = 1 + cS * b0 * xqA, cS * b0 * q1, cS * fiT * xqA, cS * fiT * q1
    assert np.allclose((J2 * x1 + J1) * x1 + J0, j1, rtol=1e-13, atol=1e-13)
    assert np.allclose(((F3 * x1 + F2) * x1 + F1) * x1 + F0, shak, rtol=1e-13, atol=1e-13)


def test_double_float_split_of_a_sum_is_exact():
    rng = np.random.default_rng(7)
    s = rng.normal(size=10000) * np.exp(rng.uniform(-20, 20, size=10000))
    hi = s.astype(np.float32)
    lo = (s - hi.astype(np.float64)).astype(np.float32)
    # hi = fl(s), lo = fl(s - hi): their sum is s to ~2^-48 relative, and hi is fl(hi + lo)
    assert np.max(np.abs((hi.astype(np.float64) + lo.astype(np.float64)) - s) / np.abs(s)) < 2.0 ** -47
    assert np.array_equal((hi.astype(np.float64) + lo.astype(np.float64)).astype(np.float32), hi)
