"""The allocation-free moment entry point (fdlb_moments_noalloc) against the solver's own
moments (fdlb_get_moments) and the FP64 oracle's moments of the same populations, on two calls
in a row with different states.  It serves callers that cannot allocate device memory (plugins in
an application that owns the whole device budget, loops that cannot take cudaMalloc's implicit
synchronisation); its scratch is a fixed array of the library, shared by all calls.  This file is
collected last on purpose."""
import numpy as np
import pytest

from oracle import solver as osolver

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb

from .cases import oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_no_alloc_moments_match_solver_moments_on_two_calls(precision):
    import torch

    fbuild.build()
    d = small_case(precision=precision, n_cells=45, Q=(4, 3, 5))
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    N = d["n_cells"]
    tsize = 4 if precision == "fp32" else 8
    f_dev = torch.empty(S.raw_elements() * tsize, dtype=torch.uint8, device="cuda")
    out = torch.empty((N, fdlb.NMOM), dtype=torch.float64, device="cuda")
    stream = S.stream_handle()
    for call, seed in enumerate((31, 32)):
        f = perturbed_state(P, seed, 0.3)
        S.set_f(f)
        expected = S.moments()
        m_or = osolver.moments(f, P)
        oracle = {"n": m_or["n"], "T": m_or["T"], "P12": m_or["P01"]}
        for a in range(3):
            oracle[f"u{a + 1}"] = m_or["u"][:, a]
            oracle[f"q{a + 1}"] = m_or["q"][:, a]
        S.get_state_raw(f_dev.data_ptr(), on_device=True)
        fdlb.moments_noalloc(precision, 4, 3, 5, N, f_dev.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, name in enumerate(fdlb.MOMENT_NAMES):
            ref = expected[name]
            scale = max(np.max(np.abs(ref)), 1e-30) if name not in ("u1", "u2", "u3", "q1", "q2", "q3", "P12") \
                else max(np.max(np.abs(expected["n"])), 1.0)
            assert np.max(np.abs(got[:, i] - ref)) <= TOL[precision] * scale, (call, name)
            assert np.max(np.abs(got[:, i] - oracle[name])) <= TOL[precision] * scale, (call, name, "oracle")


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    import torch

    fbuild.build()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(fdlb.FdlbError):
        fdlb.moments_noalloc("fp64", 2, 2, 2, 32769, x.data_ptr(), x.data_ptr())
