"""The precision pattern at steady state: FP32 populations reach a steady state on the FP32
rounding floor, some 1e-5 to 1e-4 of the moment scales away from the FP64 one for dense, small-Kn
instances; the library's two-precision schedule (fdlb_run_to_steady_mixed: FP32 to the
tolerance, then an FP64 polish on the device) brings every moment within 1e-5 of the FP64 steady
state.  The reference is the FP64 form run ten times below the compared runs' tolerance.
Instances: members of the batched-sweep distribution (seed 3) at 16 cells per sigma on the
reduced quadrature (Q = 4).  Of its first sixteen, seven converge to 1e-13 at this resolution in
FP64; the others settle on a small self-sustained oscillation of the residual (1e-10 .. 1e-7) or
converge slowly at 800+ cells.  Six of the seven are used, among them the two densest (eta0 = 0.17
and 0.23 at Kn = 0.036 and 0.023); any that would not reach the reference tolerance on another
build is left out, and at least four must remain."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import workloads as wl

from oracle import model as omodel

from .cases import accept_kn, compare_moments, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _instances():
    sweep = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e), n=16, seed=3, n_lo=64, n_hi=64)
    ds = []
    for q in (1, 2, 4, 6, 8, 9):
        d = dict(sweep[q])
        d.update(Q_R=4, Q_2=4, Q_3=4, precision="fp64",
                 n_cells=max(64, int(np.ceil(16 * omodel.confinement(d["Kn"], d["eta0"])))))
        ds.append(d)
    return ds


def test_fp32_with_fp64_polish_matches_fp64_steady_state():
    ds = _instances()
    R = fdlb.Solver(ds)
    _, _, res = R.run_to_steady(tol=1e-10, max_steps=200_000, check_every=500)
    keep = [q for q in range(len(ds)) if res[q] <= 1e-10]
    assert len(keep) >= 4, res
    ref = {q: R.moments(q) for q in keep}
    R.close()
    ds = [ds[q] for q in keep]
    F = fdlb.Solver([dict(d, precision="fp32") for d in ds])
    rc32, st32, st64, res_m = F.run_to_steady_mixed(tol=1e-9, max_steps=300_000, check_every=500)
    assert rc32 == 0 and np.all(res_m <= 1e-9), (rc32, res_m)
    assert np.all(st32 > 0) and np.all(st64 > 0)
    P32 = fdlb.Solver([dict(d, precision="fp32") for d in ds])
    P32.run_to_steady(tol=1e-8, max_steps=300_000, check_every=500)
    for j, (q, d) in enumerate(zip(keep, ds)):
        P = oracle_problem(d)
        m = ref[q]
        mo = {"n": m["n"], "T": m["T"], "P01": m["P12"], "u": np.stack([m[f"u{a + 1}"] for a in range(3)], -1),
              "q": np.stack([m[f"q{a + 1}"] for a in range(3)], -1)}
        err_mixed = compare_moments(F.moments(j), mo, P)
        err_fp32 = compare_moments(P32.moments(j), mo, P)
        print("instance", q, "FP32 alone", err_fp32, "FP32 + FP64 polish", err_mixed)
        assert max(err_mixed.values()) <= 1e-5, (q, err_mixed)
