"""Large half-range orders on the radial axis (the paper's HHLB(7,20), HHLB(7,60) and HHLB(7,100),
Sec. IV): 2Q_R = 40 .. 200 radial momenta, where the K^h contraction of the curvature force runs as
its own kernel and the fused stage reads its result.  The right-hand side and a few steps against
the FP64 oracle on the same seeded inputs, in both precisions."""
import numpy as np
import pytest

from oracle import solver as osolver
from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import workloads as wl

from .cases import compare_moments, oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}
RHS_TOL = {"fp64": 1e-10, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


CASES = [  # (geometry, Q_R, Q_2, Q_3, cells)
    (wl.CYL, 20, 8, 8, 29), (wl.CYL, 50, 4, 4, 23), (wl.CYL, 100, 4, 4, 17), (wl.SPH, 20, 8, 8, 21),
    (wl.CYL, 16, 6, 4, 33),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("geom,QR,Q2,Q3,N", CASES)
def test_large_radial_order_rhs_and_steps_match_oracle(precision, geom, QR, Q2, Q3, N):
    d = small_case(geometry=geom, precision=precision, n_cells=N, Q=(QR, Q2, Q3), beta=0.8, Kn=0.05, eta0=0.15)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 17, 0.05)
    S = fdlb.Solver(d)
    S.set_f(f0)
    L = S.eval_rhs()
    L_or = osolver.rhs(f0, P)
    err = np.max(np.abs(L - L_or)) / np.max(np.abs(L_or))
    assert err <= RHS_TOL[precision], err
    S.step(4)
    f_or = osolver.run(f0, P, 4)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL[precision], errs


def test_paper_couette_quadrature_hhlb_7_20():
    """Cylindrical Couette flow on the paper's quadrature HHLB(7,20) x HLB(7,8) x HLB(7,8) (the
    dense cases of Sec. IV.A: eta0 = 0.1, C = 4, R_L = 1, sigma = 1, inner wall at U_w = sqrt(T_w)),
    FP32, 30 steps from the uniform start against the oracle."""
    d = dict(geometry=wl.CYL, R_in=1.0, R_out=5.0, sigma=1.0, n_cells=40, beta=0.0, Q_R=20, Q_2=8, Q_3=8,
             eta0=0.1, T_wall=(1.0, 1.0), u_wall=(1.0, 0.0), dt=None, precision="fp32", chi_model=0)
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    S.step(30)
    f_or = osolver.run(osolver.uniform_state(P), P, 30)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs


@pytest.mark.parametrize("QR", [16, 20, 50, 100])
def test_tensor_core_contraction_matches_cuda_core_kernel(QR):
    """The tcgen05 split-TF32 contraction kernel against the CUDA-core kernel on the same state
    (FP32 populations; 19 cells x 4 values of p_3 x 8 of p_2 per tile column block, so the last
    tile of 128 columns is partial)."""
    d = small_case(precision="fp32", n_cells=19, Q=(QR, 8, 4), beta=0.5, Kn=0.05, eta0=0.15)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 29, 0.1)
    S = fdlb.Solver(d)
    S.set_f(f0)
    assert S.set_tensor_contraction(True)
    L_tc = S.eval_rhs()
    assert not S.set_tensor_contraction(False)
    L_cc = S.eval_rhs()
    assert np.max(np.abs(L_tc - L_cc)) <= 2e-6 * np.max(np.abs(L_cc))
    rc = S.diagnostics()[0]
    assert rc == 0
