"""The learned warm start end to end at reduced scale: steady states of seeded sweep instances
computed by the solver, the network trained on them with the library's kernels, and the
SSP-RK3 steps to the residual tolerance on held-out instances with and without the network."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import warmstart as ws
from paper_2403_15051_gb300 import workloads as wl

from .cases import accept_kn

pytestmark = pytest.mark.gpu


def _instances(n, seed):
    ds = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e) and kn >= 0.05, n=n, seed=seed, n_lo=48, n_hi=48)
    for d in ds:
        d.update(Q_R=4, Q_2=4, Q_3=4)
    return ds


def test_trained_network_reduces_steps_to_steady():
    fbuild.build()
    P = 64
    train_ds, eval_ds = _instances(48, 101), _instances(12, 202)
    raw, tg, steps, res, rc = ws.steady_states(train_ds, n_points=P, tol=1e-6, max_steps=60_000, check_every=100)
    assert rc == 0, (rc, res)
    net, losses = ws.train(raw, tg, epochs=300, batch=16, lr=2e-3, width=32, modes=6, layers=3, hidden=64)
    assert losses[-1] < 0.2 * losses[0]
    # the seed carries each instance's own total mass (the walls conserve it)
    S = fdlb.Solver(eval_ds)
    m_uniform = [S.diagnostics(q)[1] for q in range(len(eval_ds))]
    for q, d in enumerate(eval_ds):
        net.warm_start(S, q, ws.raw_parameters(d))
    m_seed = [S.diagnostics(q)[1] for q in range(len(eval_ds))]
    S.close()
    assert np.allclose(m_seed, m_uniform, rtol=1e-5), (m_seed, m_uniform)
    cold, _, rc1 = ws.steps_to_steady(eval_ds, None, tol=1e-6, max_steps=60_000, check_every=100)
    warm, _, rc2 = ws.steps_to_steady(eval_ds, net, tol=1e-6, max_steps=60_000, check_every=100)
    assert rc1 == 0 and rc2 == 0
    print("steps uniform", cold, "warm", warm)
    assert np.mean(warm) < 0.8 * np.mean(cold)
