"""Learned warm start: training data from the solver's own steady states, training with the
library's network kernels, and the steps-to-steady comparison against the uniform start.

All numerical work runs in libfdlb_gb300.so (solver kernels, network forward/backward/Adam
kernels); this module only moves arrays between those calls:

* `steady_states(ds)`: one batched handle, `fdlb_run_to_steady`, per-cell moments sampled at
  P points of the normalised radius and encoded as the network's targets
  (n/n0 - 1, u_2/0.1, (T/T_in - 1)/0.1, q_R/(0.01 n0 T_in^1.5), as in include/fdlb.h);
* `train(...)`: minibatch Adam through `fdlb_nn_train_step`;
* `steps_to_steady(ds, net)`: SSP-RK3 steps to the residual tolerance from the uniform start or
  from the network's prediction (`fdlb_nn_warm_start`), in one batched handle.
"""
from __future__ import annotations

import numpy as np

from . import fdlb


def raw_parameters(d):
    """(Kn, eta0, R_out/R_in, inner wall speed, T_out/T_in) of a workload dictionary."""
    return np.array([d["Kn"], d["eta0"], d["R_out"] / d["R_in"], d["u_wall"][0], d["T_wall"][1] / d["T_wall"][0]],
                    dtype=np.float32)


def encode_profiles(S, q, n_points):
    """Moments of instance q sampled at n_points equally spaced points of the normalised radius
    (linear interpolation between cell centres), encoded as the network's output channels."""
    inf = S.info(q)
    d = S.param_dicts[q]
    Rc, Rf, _, _ = fdlb.grid(d["geometry"], d["R_in"], d["R_out"], inf["sigma"], d["n_cells"], d.get("beta") or 0.0)
    xc = (Rc - Rf[0]) / (Rf[-1] - Rf[0])
    x = np.linspace(0.0, 1.0, n_points)
    m = S.moments(q)
    Tin = d["T_wall"][0]
    n0 = inf["n0"]
    ch = [np.interp(x, xc, m["n"]) / n0 - 1.0, np.interp(x, xc, m["u2"]) / 0.1,
          (np.interp(x, xc, m["T"]) / Tin - 1.0) / 0.1, np.interp(x, xc, m["q1"]) / (0.01 * n0 * Tin ** 1.5)]
    return np.stack(ch, axis=-1).astype(np.float32)


def steady_states(ds, n_points=256, tol=1e-8, max_steps=400_000, check_every=200, stall_checks=0):
    """Run every instance to steady state in one batched handle; returns (raw [M][5],
    targets [M][P][4], steps [M], residuals [M], status).  stall_checks: the library's stall rule
    (instances whose residual has stopped falling stop stepping; 0: off)."""
    S = fdlb.Solver(ds)
    S.set_stall_checks(stall_checks)
    rc, steps, res = S.run_to_steady(tol=tol, max_steps=max_steps, check_every=check_every)
    raw = np.stack([raw_parameters(d) for d in ds])
    tg = np.stack([encode_profiles(S, q, n_points) for q in range(len(ds))])
    S.close()
    return raw, tg, steps, res, rc


def train(raw, targets, epochs=400, batch=32, lr=1e-3, seed=0, width=64, modes=6, layers=4, hidden=128):
    """Minibatch Adam on (raw, targets) with a cosine learning-rate decay; returns the network
    and the per-epoch mean loss."""
    net = fdlb.WarmStartNet(width, modes, layers, hidden, targets.shape[1], max_batch=batch)
    net.init_params(seed)
    rng = np.random.default_rng(seed)
    M = raw.shape[0]
    losses = []
    for ep in range(epochs):
        lr_ep = 0.5 * lr * (1.0 + np.cos(np.pi * ep / epochs))
        perm = rng.permutation(M)
        tot = 0.0
        for s0 in range(0, M, batch):
            idx = perm[s0:s0 + batch]
            tot += net.train_step(raw[idx], targets[idx], lr_ep) * len(idx)
        losses.append(tot / M)
    return net, losses


def steps_to_steady(ds, net=None, tol=1e-8, max_steps=400_000, check_every=200, stall_checks=0):
    """SSP-RK3 steps to the residual tolerance, from the uniform equilibrium (net None) or from
    the network's predicted profiles."""
    S = fdlb.Solver(ds)
    S.set_stall_checks(stall_checks)
    if net is not None:
        for q, d in enumerate(ds):
            net.warm_start(S, q, raw_parameters(d))
    rc, steps, res = S.run_to_steady(tol=tol, max_steps=max_steps, check_every=check_every)
    S.close()
    return steps, res, rc
