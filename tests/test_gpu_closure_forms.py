"""The two forms of the closure give the same collision records, hence the same populations, bit
for bit: the item chain (one launch; a block takes an item of a few cells through the whole
closure) and the batch form (two launches over items of 28 cells: every cell's n, u, T, q and FM
band sum, then the records of each item from the fields of its reach).  Ragged item counts, both
geometries and precisions, chi at the local density, the cylinder with p_z integrated out, a batch
of sweep instances of different lengths."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import workloads as wl

from .cases import accept_kn, oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _run(ds, form, states, steps):
    S = fdlb.Solver(ds)
    S.set_autotune(0)
    assert S.closure_form(form) == form
    for q, f0 in enumerate(states):
        S.set_f(f0, q)
    S.step(steps)
    out = [S.get_f(q) for q in range(len(ds))], [S.closure(q) for q in range(len(ds))]
    S.close()
    return out


def _check(ds, steps=12, seed=5):
    states = [perturbed_state(oracle_problem(d), seed + q, 0.05) for q, d in enumerate(ds)]
    fa, ca = _run(ds, 0, states, steps)
    fb, cb = _run(ds, 1, states, steps)
    for q in range(len(ds)):
        assert np.all(np.isfinite(fa[q]))
        assert np.array_equal(fa[q], fb[q]), (q, np.max(np.abs(fa[q] - fb[q])))
        for k in ca[q]:
            assert np.array_equal(ca[q][k], cb[q][k]), (q, k)


CASES = {
    "cyl-fp32": dict(geometry=wl.CYL, precision="fp32", n_cells=61, u_wall=(0.2, 0.0)),
    "cyl-fp64-stretched": dict(geometry=wl.CYL, precision="fp64", n_cells=57, beta=1.5),
    "sph-fp32": dict(geometry=wl.SPH, precision="fp32", n_cells=59, beta=1.2),
    "sph-fp64": dict(geometry=wl.SPH, precision="fp64", n_cells=30),
    "cyl-fp32-chi-local": dict(geometry=wl.CYL, precision="fp32", n_cells=45, chi_model=fdlb.CHI_SET_LOCAL),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_closure_forms_agree(name):
    _check([small_case(**CASES[name])])


def test_closure_forms_agree_reduced_cylinder():
    d = wl.couette_cyl_reduced(Q_R=4, Q_2=4, cells_per_sigma=10)
    _check([d])


def test_closure_forms_agree_on_a_batch():
    ds = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e), n=5, seed=2, n_lo=20, n_hi=90)
    for d in ds:
        d.update(Q_R=4, Q_2=4, Q_3=4)
    _check(ds, steps=9)


def test_batch_form_is_the_default_for_many_items():
    ds = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e), n=64, seed=0, n_lo=128, n_hi=512)
    for d in ds:
        d.update(Q_R=2, Q_2=2, Q_3=2)
    S = fdlb.Solver(ds)
    assert S.closure_form() == 1
    S.close()
    T = fdlb.Solver(small_case(n_cells=40))
    assert T.closure_form() == 0
    T.close()
