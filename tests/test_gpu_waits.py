"""Failure detection of the bounded device waits, without a GPU fault: a test hook makes a wait
run out (a copy barrier expecting bytes that never arrive; a grid barrier expecting arrivals that
never come); the blocks set the error flag and leave, the host reads FDLB_ETIMEOUT, and after the
flag is cleared the same handle steps on and matches a fresh one bit for bit."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb

from .cases import oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _recover_and_compare(S, d, f0, persistent):
    S.set_wait_test(0, 0)
    S.clear_error()
    S.set_f(f0)
    S.step(3)
    rc, _, _, _ = S.diagnostics()
    assert rc == 0
    R = fdlb.Solver(d)
    R.set_persistent_step(persistent)
    R.set_f(f0)
    R.step(3)
    assert np.array_equal(S.get_f(), R.get_f())


def test_staged_copy_wait_runs_out_and_is_reported():
    d = small_case(precision="fp32", n_cells=16)
    f0 = perturbed_state(oracle_problem(d), 4, 0.05)
    S = fdlb.Solver(d)
    S.set_f(f0)
    S.set_wait_test(tx_extra_bytes=16)
    S.eval_rhs()  # one stage: its copy barriers run out (1 s), its result is undefined
    rc, _, _, _ = S.diagnostics()
    assert rc == ETIMEOUT
    _recover_and_compare(S, d, f0, False)


def test_grid_barrier_wait_runs_out_and_is_reported():
    d = small_case(precision="fp32", n_cells=32, Q=(8, 8, 8))
    f0 = perturbed_state(oracle_problem(d), 6, 0.05)
    S = fdlb.Solver(d)
    assert S.set_persistent_step(True)
    S.set_f(f0)
    S.set_wait_test(barrier_extra=1)
    S.step(1)
    rc, _, _, _ = S.diagnostics()
    assert rc == ETIMEOUT
    _recover_and_compare(S, d, f0, True)
