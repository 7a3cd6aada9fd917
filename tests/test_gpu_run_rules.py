"""Stopping rules of fdlb_run_to_steady in a batch: an instance whose moments become non-finite
stops alone (residual +inf, status FDLB_ENAN) while the others run on to the tolerance; with the
stall rule an instance whose residual has stopped falling stops unconverged instead of holding
the batch to max_steps; the FP32-then-FP64 mode carries both through its two phases."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb

from .cases import small_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _batch(precision):
    return [small_case(precision=precision, n_cells=n, Kn=kn, eta0=e, T_wall=(1.0, t), u_wall=(u, 0.0), R=(1.0, r),
                       Q=(4, 4, 4))
            for n, kn, e, t, u, r in ((24, 0.2, 0.05, 1.1, 0.1, 2.0), (30, 0.3, 0.1, 1.2, 0.0, 3.0),
                                      (20, 0.25, 0.08, 1.0, 0.2, 1.5))]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_a_non_finite_instance_stops_alone(precision):
    ds = _batch(precision)
    S = fdlb.Solver(ds)
    bad = S.get_f(1)
    bad[2, 0, 0, 0] = np.nan
    S.set_f(bad, 1)
    rc, steps, res = S.run_to_steady(tol=1e-8, max_steps=200_000, check_every=200)
    assert rc == 6  # FDLB_ENAN
    assert np.isinf(res[1]) and steps[1] == 200
    assert res[0] <= 1e-8 and res[2] <= 1e-8, res
    # the clean instances reached the same steady states as on their own
    for q in (0, 2):
        T = fdlb.Solver(ds[q])
        T.run_to_steady(tol=1e-8, max_steps=200_000, check_every=200)
        assert np.max(np.abs(T.moments()["n"] - S.moments(q)["n"])) <= 1e-6 * np.max(T.moments()["n"])


def test_stalled_instances_stop_before_max_steps():
    ds = _batch("fp64")
    S = fdlb.Solver(ds)
    S.step(500)  # past the fast relaxation of q: the residual now falls on the flow's slow scale
    # checks ten steps apart: a relaxing residual does not halve between them, so with a stall
    # window of five checks every instance stops after six checks (sixty steps), unconverged
    S.set_stall_checks(5)
    rc, steps, res = S.run_to_steady(tol=1e-30, max_steps=10_000, check_every=10)
    assert rc == 4  # FDLB_ENOTCONVERGED
    assert np.all(steps == 60) and np.all(res > 1e-30), (steps, res)
    S.set_stall_checks(0)
    rc, steps, _ = S.run_to_steady(tol=1e-30, max_steps=100, check_every=10)
    assert rc == 4 and np.all(steps == 100)
    with pytest.raises(fdlb.FdlbError):
        S.set_stall_checks(-1)


def test_mixed_mode_carries_the_stopping_rules():
    ds = _batch("fp32")
    S = fdlb.Solver(ds)
    bad = S.get_f(0)
    bad[1, 0, 0, 0] = np.inf
    S.set_f(bad, 0)
    rc, s32, s64, res = S.run_to_steady_mixed(tol=1e-9, max_steps=200_000, check_every=200)
    assert rc == 6
    assert not np.isfinite(res[0]) and np.all(res[1:] <= 1e-9), res
