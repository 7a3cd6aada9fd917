"""FP64 reference of the learned warm-start network: a one-dimensional Fourier neural operator
mapping the five instance parameters (Kn, eta0, radius ratio, wall speed, temperature ratio) to
four moment profiles on P points of the normalised radius.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Gradients are written out by hand
(reverse mode), so the tests can pin them against finite differences and then against the
GPU's training kernels.

Architecture (all sizes are arguments):
    a[b, x]   = [features of the 5 parameters, x / (P - 1)]                      (cin = 6)
    v0        = a Wlift + blift                                                  (width W)
    v_{l+1}   = GELU(v_l W_l + b_l + S_l(v_l)),  l = 0..L-1
    S_l(v)    = G [ R_l (F v) ]      F: 2m x P real DFT rows (cos, -sin) of the m lowest modes,
                                     R_l: per-mode complex W x W mixing, G: truncated inverse
    h         = GELU(v_L P1 + c1)                                                (hidden H)
    out       = h P2 + c2                                                        (4 outputs)
    loss      = mean((out - target)^2)
GELU(x) = x Phi(x) with Phi the standard normal distribution function.

Parameter vector layout (shared with the GPU kernels): lift W [cin][W], lift b [W]; per layer
R_re [m][W][W], R_im [m][W][W], W [W][W], b [W]; P1 [W][H], c1 [H]; P2 [H][cout], c2 [cout].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def layout(W=64, m=6, L=4, H=128, cin=6, cout=4):
    shapes = [("lift_w", (cin, W)), ("lift_b", (W,))]
    for l in range(L):
        shapes += [(f"r_re{l}", (m, W, W)), (f"r_im{l}", (m, W, W)), (f"w{l}", (W, W)), (f"b{l}", (W,))]
    shapes += [("p1_w", (W, H)), ("p1_b", (H,)), ("p2_w", (H, cout)), ("p2_b", (cout,))]
    out, off = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out, off


def unpack(theta, lay):
    return {k: theta[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in lay.items()}


def dft_matrices(P, m):
    """F [2m][P]: rows cos(2 pi k x / P) then -sin(2 pi k x / P), k = 0..m-1; G [P][2m]: the
    truncated inverse, y[x] = (1/P) sum_k c_k (Yre_k cos - Yim_k sin), c_0 = 1, c_k = 2."""
    x = np.arange(P)
    k = np.arange(m)
    ang = 2.0 * math.pi * np.outer(k, x) / P
    F = np.concatenate([np.cos(ang), -np.sin(ang)], axis=0)
    c = np.where(k == 0, 1.0, 2.0)
    G = np.concatenate([(c[:, None] * np.cos(ang)).T, (c[:, None] * -np.sin(ang)).T], axis=1) / P
    return F, G


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def features(pfeat, P):
    """[B][P][6]: the five (already normalised) parameters broadcast over x, then x/(P-1)."""
    B = pfeat.shape[0]
    a = np.empty((B, P, pfeat.shape[1] + 1))
    a[:, :, :-1] = pfeat[:, None, :]
    a[:, :, -1] = np.arange(P) / (P - 1)
    return a


def forward(theta, pfeat, P=256, W=64, m=6, L=4, H=128):
    lay, _ = layout(W, m, L, H)
    p = unpack(theta, lay)
    F, G = dft_matrices(P, m)
    a = features(pfeat, P)
    cache = {"a": a, "vs": [], "us": [], "vhat": []}
    v = a @ p["lift_w"] + p["lift_b"]
    for l in range(L):
        vh = np.einsum("kx,bxc->bkc", F, v)  # [B][2m][W]
        re, im = vh[:, :m], vh[:, m:]
        yre = np.einsum("bki,kio->bko", re, p[f"r_re{l}"]) - np.einsum("bki,kio->bko", im, p[f"r_im{l}"])
        yim = np.einsum("bki,kio->bko", re, p[f"r_im{l}"]) + np.einsum("bki,kio->bko", im, p[f"r_re{l}"])
        s = np.einsum("xk,bkc->bxc", G, np.concatenate([yre, yim], axis=1))
        u = v @ p[f"w{l}"] + p[f"b{l}"] + s
        cache["vs"].append(v)
        cache["vhat"].append(vh)
        cache["us"].append(u)
        v = gelu(u)
    z1 = v @ p["p1_w"] + p["p1_b"]
    h = gelu(z1)
    out = h @ p["p2_w"] + p["p2_b"]
    cache.update(vL=v, z1=z1, h=h, F=F, G=G)
    return out, cache


def backward(theta, cache, dout, P=256, W=64, m=6, L=4, H=128):
    lay, n = layout(W, m, L, H)
    p = unpack(theta, lay)
    g = {k: np.zeros(s) for k, (o, s) in lay.items()}
    F, G = cache["F"], cache["G"]
    g["p2_w"] = np.einsum("bxh,bxo->ho", cache["h"], dout)
    g["p2_b"] = dout.sum((0, 1))
    dh = dout @ p["p2_w"].T
    dz1 = dh * gelu_grad(cache["z1"])
    g["p1_w"] = np.einsum("bxw,bxh->wh", cache["vL"], dz1)
    g["p1_b"] = dz1.sum((0, 1))
    dv = dz1 @ p["p1_w"].T
    for l in reversed(range(L)):
        u, v, vh = cache["us"][l], cache["vs"][l], cache["vhat"][l]
        du = dv * gelu_grad(u)
        g[f"w{l}"] = np.einsum("bxi,bxo->io", v, du)
        g[f"b{l}"] = du.sum((0, 1))
        dv = du @ p[f"w{l}"].T
        # spectral part: s = G [yre; yim]
        dy = np.einsum("xk,bxc->bkc", G, du)
        dyre, dyim = dy[:, :m], dy[:, m:]
        re, im = vh[:, :m], vh[:, m:]
        g[f"r_re{l}"] = np.einsum("bki,bko->kio", re, dyre) + np.einsum("bki,bko->kio", im, dyim)
        g[f"r_im{l}"] = np.einsum("bki,bko->kio", re, dyim) - np.einsum("bki,bko->kio", im, dyre)
        dre = np.einsum("bko,kio->bki", dyre, p[f"r_re{l}"]) + np.einsum("bko,kio->bki", dyim, p[f"r_im{l}"])
        dim = -np.einsum("bko,kio->bki", dyre, p[f"r_im{l}"]) + np.einsum("bko,kio->bki", dyim, p[f"r_re{l}"])
        dv = dv + np.einsum("kx,bkc->bxc", F, np.concatenate([dre, dim], axis=1))
    g["lift_w"] = np.einsum("bxi,bxw->iw", cache["a"], dv)
    g["lift_b"] = dv.sum((0, 1))
    grad = np.zeros(n)
    for k, (o, s) in lay.items():
        grad[o:o + int(np.prod(s))] = g[k].ravel()
    return grad


def loss_and_grad(theta, pfeat, target, **kw):
    out, cache = forward(theta, pfeat, **kw)
    diff = out - target
    loss = float(np.mean(diff * diff))
    dout = 2.0 * diff / diff.size
    return loss, backward(theta, cache, dout, **kw), out


def init_params(seed, W=64, m=6, L=4, H=128, cin=6, cout=4):
    """Seeded initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)); spectral weights scaled
    by 1/(W W)."""
    lay, n = layout(W, m, L, H, cin, cout)
    rng = np.random.default_rng(seed)
    theta = np.zeros(n)
    for k, (o, s) in lay.items():
        size = int(np.prod(s))
        if k.startswith("r_"):
            theta[o:o + size] = rng.uniform(0.0, 1.0, size) / (W * W)
        elif k.endswith("_b") or (k[0] == "b" and k[1:].isdigit()):
            theta[o:o + size] = 0.0
        else:
            fan_in = s[0]
            theta[o:o + size] = rng.uniform(-1.0, 1.0, size) / math.sqrt(fan_in)
    return theta
