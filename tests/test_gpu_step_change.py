"""The per-step change of the populations (fdlb_step_change), the second convergence measure beside
the moment residual: it matches the change computed from the states before and after the step, and
it vanishes as an FP64 state reaches its steady state."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb

from .cases import oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_change_matches_the_states(precision):
    ds = [small_case(precision=precision, n_cells=n, Q=(4, 4, 4), Kn=kn) for n, kn in ((24, 0.1), (37, 0.05))]
    S = fdlb.Solver(ds)
    for q, d in enumerate(ds):
        S.set_f(perturbed_state(oracle_problem(d), 3 + q, 0.05), q)
    before = [S.get_f(q).astype(np.float64) for q in range(len(ds))]
    rel = S.step_change()
    for q in range(len(ds)):
        after = S.get_f(q).astype(np.float64)
        ref = np.linalg.norm(after - before[q]) / np.linalg.norm(before[q])
        assert rel[q] == pytest.approx(ref, rel=1e-9), (q, rel[q], ref)
        assert rel[q] > 0.0


def test_step_change_vanishes_at_an_fp64_steady_state():
    d = small_case(precision="fp64", n_cells=24, Q=(4, 4, 4), Kn=0.2, eta0=0.05, T_wall=(1.0, 1.1), u_wall=(0.1, 0.0))
    S = fdlb.Solver(d)
    first = S.step_change()[0]
    S.run_to_steady(tol=1e-12, max_steps=400_000, check_every=200)
    last = S.step_change()[0]
    assert first > 1e-6 and last < 1e-10, (first, last)
