"""The cylinder with p_z integrated out (FDLB_CYL_Z; the reduced pair phi = int f dp_z,
chi = int p_z^2 f dp_z of Sec. III.A's remark on Couette flow) against the oracle's reduced model:
the right-hand side and twenty steps in both precisions, mass conservation, the warm-start seed,
and Couette flow on the paper's own quadrature HHLB(7,20) x HLB(7,8)."""
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


def _case(precision, n_cells=37, Q=(6, 8), **kw):
    d = small_case(precision=precision, n_cells=n_cells, Q=(Q[0], Q[1], 0), beta=0.9, **kw)
    d["geometry"] = wl.CYL_Z
    return d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chi_model", [0, 1])
def test_reduced_rhs_and_twenty_steps_match_oracle(precision, chi_model):
    d = _case(precision, chi_model=chi_model)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 31, 0.05)
    S = fdlb.Solver(d)
    assert S.info()["n_momenta"] == 2 * 12 * 8
    S.set_f(f0)
    L_or, det = osolver.rhs(f0, P, details=True)
    L = S.eval_rhs()
    assert np.max(np.abs(L - L_or)) / np.max(np.abs(L_or)) <= RHS_TOL[precision]
    cl = S.closure()
    assert np.allclose(cl["n_wall"], det["n_wall"], rtol=1e-11 if precision == "fp64" else 1e-5)
    S.step(20)
    f_or = osolver.run(f0, P, 20)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL[precision], errs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_reduced_mass_conservation_and_seed(precision):
    d = _case(precision, n_cells=40)
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    xp = np.linspace(0.0, 1.0, 17)
    prof = [P.n0 * (1 + 0.1 * xp), 0.15 * xp, 1.0 + 0.2 * xp, 0.02 * P.n0 * np.cos(3 * xp)]
    S.init_from_moments(0, *prof)
    xc = (P.grid.R_c - P.grid.R_f[0]) / (P.grid.R_f[-1] - P.grid.R_f[0])
    f_or = osolver.shakhov_seed(P, *[np.interp(xc, xp, v) for v in prof])
    assert np.max(np.abs(S.get_f() - f_or)) <= (1e-12 if precision == "fp64" else 1e-6) * np.max(np.abs(f_or))
    m0 = S.diagnostics()[1]
    assert m0 == pytest.approx(osolver.total_mass(f_or, P), rel=1e-12 if precision == "fp64" else 1e-6)
    S.step(300)
    rc, m1, _, _ = S.diagnostics()
    assert rc == 0 and abs(m1 - m0) / m0 <= (1e-12 if precision == "fp64" else 2e-5)


def test_reduced_paper_quadrature_couette():
    """The paper's cylindrical Couette set-up (eta0 = 0.1, C = 4, R_L = 1, U_w = sqrt(T_w)) on its
    quadrature HHLB(7,20) x HLB(7,8) with p_z integrated out (40 x 8 x 2 = 640 populations per cell),
    FP32: thirty steps against the oracle; the K^h contraction runs as its own kernel."""
    d = wl.couette_cyl_reduced()
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    S.step(30)
    f_or = osolver.run(osolver.uniform_state(P), P, 30)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs
