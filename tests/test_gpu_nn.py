"""The warm-start network's GPU kernels (BF16 weights, FP32 accumulation) against the FP64 oracle
network: forward outputs, loss and every gradient; and training reduces the loss."""
import numpy as np
import pytest

from oracle import nn as onn
from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def normalise(raw):
    """The network's input encoding (fdlb_nn_* in include/fdlb.h)."""
    return np.stack([np.log10(raw[:, 0]) + 1.0, (raw[:, 1] - 0.155) / 0.145, (raw[:, 2] - 3.1) / 1.9,
                     (raw[:, 3] - 0.15) / 0.15, (raw[:, 4] - 1.15) / 0.15], axis=1)


def raw_params(B, seed):
    rng = np.random.default_rng(seed)
    return np.stack([10 ** rng.uniform(-2, 0, B), rng.uniform(0.01, 0.3, B), rng.uniform(1.2, 5, B),
                     rng.uniform(0, 0.3, B), rng.uniform(1.0, 1.3, B)], axis=1).astype(np.float32)


@pytest.mark.parametrize("sizes", [dict(W=16, m=4, L=2, H=32, P=64), dict(W=64, m=6, L=4, H=128, P=256)])
def test_forward_loss_and_gradients_match_fp64_oracle(sizes):
    fbuild.build()
    B = 4
    theta = bf16_round(onn.init_params(3, W=sizes["W"], m=sizes["m"], L=sizes["L"], H=sizes["H"]))
    # give the spectral weights and biases a size at which every term contributes
    lay, _ = onn.layout(sizes["W"], sizes["m"], sizes["L"], sizes["H"])
    rng = np.random.default_rng(5)
    for k, (o, s) in lay.items():
        n = int(np.prod(s))
        if k.startswith("r_"):
            theta[o:o + n] = bf16_round(rng.normal(0, 0.5 / sizes["W"], n))
        if k.endswith("_b") or (k[0] == "b" and k[1:].isdigit()):
            theta[o:o + n] = bf16_round(rng.normal(0, 0.1, n))
    raw = raw_params(B, 11)
    target = np.random.default_rng(12).normal(0, 1, (B, sizes["P"], 4)).astype(np.float32)
    net = fdlb.WarmStartNet(sizes["W"], sizes["m"], sizes["L"], sizes["H"], sizes["P"], max_batch=8)
    assert net.n_params == theta.size
    net.set_params(theta.astype(np.float32))
    kw = dict(P=sizes["P"], W=sizes["W"], m=sizes["m"], L=sizes["L"], H=sizes["H"])
    pfeat = normalise(raw.astype(np.float64))
    loss_o, grad_o, out_o = onn.loss_and_grad(theta, pfeat, target.astype(np.float64), **kw)
    out = net.forward(raw)
    assert np.max(np.abs(out - out_o)) <= 2e-4 * max(1.0, np.max(np.abs(out_o)))
    loss, grad = net.loss_grad(raw, target)
    assert loss == pytest.approx(loss_o, rel=1e-4)
    for k, (o, s) in lay.items():
        n = int(np.prod(s))
        go, gg = grad_o[o:o + n], grad[o:o + n]
        scale = max(np.max(np.abs(go)), 1e-12)
        assert np.max(np.abs(gg - go)) <= 2e-3 * scale, k


def test_training_reduces_the_loss():
    fbuild.build()
    sizes = dict(W=32, m=6, L=2, H=64, P=128)
    net = fdlb.WarmStartNet(sizes["W"], sizes["m"], sizes["L"], sizes["H"], sizes["P"], max_batch=32)
    net.set_params(onn.init_params(1, W=sizes["W"], m=sizes["m"], L=sizes["L"], H=sizes["H"]).astype(np.float32))
    raw = raw_params(32, 21)
    x = np.linspace(0, 1, sizes["P"])
    f = normalise(raw.astype(np.float64))
    # a smooth synthetic target family of the parameters
    target = np.stack([0.3 * f[:, 0:1] * np.cos(np.pi * x), f[:, 3:4] * (1 - x), 0.5 * f[:, 4:5] * x,
                       0.2 * f[:, 1:2] * np.ones_like(x)], axis=-1).astype(np.float32)
    first = net.train_step(raw, target, 1e-3)
    for _ in range(300):
        last = net.train_step(raw, target, 1e-3)
    assert last < 0.1 * first
