"""Pins of the FP64 warm-start network oracle: the hand-written backward pass against central
finite differences, the DFT pair against numpy's FFT, and GELU against its definition."""
import math

import numpy as np
import pytest

from oracle import nn

SMALL = dict(P=32, W=8, m=3, L=2, H=16)


def _setup(seed=0, B=3):
    theta = nn.init_params(seed, W=SMALL["W"], m=SMALL["m"], L=SMALL["L"], H=SMALL["H"])
    rng = np.random.default_rng(seed + 1)
    # larger spectral weights than the default initialisation so that every term matters
    lay, _ = nn.layout(SMALL["W"], SMALL["m"], SMALL["L"], SMALL["H"])
    for k, (o, s) in lay.items():
        if k.startswith("r_"):
            theta[o:o + int(np.prod(s))] = rng.normal(0.0, 0.3, int(np.prod(s)))
        if k.endswith("b") or k[0] == "b":
            theta[o:o + int(np.prod(s))] = rng.normal(0.0, 0.1, int(np.prod(s)))
    pfeat = rng.uniform(-1, 1, (B, 5))
    target = rng.normal(0, 1, (B, SMALL["P"], 4))
    return theta, pfeat, target


def test_backward_matches_central_differences():
    theta, pfeat, target = _setup()
    loss, grad, _ = nn.loss_and_grad(theta, pfeat, target, **SMALL)
    rng = np.random.default_rng(7)
    idx = rng.choice(theta.size, 60, replace=False)
    lay, _ = nn.layout(SMALL["W"], SMALL["m"], SMALL["L"], SMALL["H"])
    # make sure every parameter group is probed at least once
    idx = np.unique(np.concatenate([idx, [o for o, _ in lay.values()]]))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = nn.loss_and_grad(tp, pfeat, target, **SMALL)[0]
        lm = nn.loss_and_grad(tm, pfeat, target, **SMALL)[0]
        fd = (lp - lm) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_dft_pair_matches_numpy_fft():
    P, m = 32, 5
    F, G = nn.dft_matrices(P, m)
    rng = np.random.default_rng(3)
    v = rng.normal(size=P)
    spec = np.fft.rfft(v)[:m]
    vh = F @ v
    assert np.allclose(vh[:m], spec.real, atol=1e-12) and np.allclose(vh[m:], spec.imag, atol=1e-12)
    # G is the inverse restricted to the kept modes: G F projects on them
    full = np.zeros(P // 2 + 1, complex)
    full[:m] = spec
    assert np.allclose(G @ vh, np.fft.irfft(full, n=P), atol=1e-12)


def test_gelu_definition():
    x = np.linspace(-5, 5, 41)
    Phi = 0.5 * (1 + np.array([math.erf(t / math.sqrt(2)) for t in x]))
    assert np.allclose(nn.gelu(x), x * Phi, atol=1e-15)
    h = 1e-6
    assert np.allclose(nn.gelu_grad(x), (nn.gelu(x + h) - nn.gelu(x - h)) / (2 * h), atol=1e-8)


def test_layout_size_of_the_full_network():
    _, n = nn.layout()
    assert 2.0e5 < n < 2.5e5  # about 2e5 parameters (4 layers, width 64)
