"""The persistent step kernel (whole SSP-RK3 steps in one cooperative launch, the closure of each
tile computed by the block that streams it, grid barriers between stages) against the closure +
stage kernels: the same populations bit for bit, on both compile-time quadratures (the 24 x 12
x 12 sphere in FP32: its FP64 rows do not fit in shared memory), with and without the FM band,
and with more tiles than blocks; and against the FP64 oracle."""
import numpy as np
import pytest

from oracle import solver as osolver
from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import workloads as wl

from .cases import compare_moments, oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _run(d, f0, persistent, steps, tiling=None):
    S = fdlb.Solver(d)
    if tiling:
        S.set_tiling(*tiling)
    used = S.set_persistent_step(persistent)
    S.set_f(f0)
    S.step(steps)
    return used, S.get_f(), S.moments()


CASES = [
    ("cyl-fp32-band", dict(geometry=wl.CYL, precision="fp32", n_cells=96, Q=(8, 8, 8), beta=1.5)),
    ("cyl-fp32-local", dict(geometry=wl.CYL, precision="fp32", n_cells=70, Q=(8, 8, 8), beta=0.0)),
    ("cyl-fp64-band", dict(geometry=wl.CYL, precision="fp64", n_cells=80, Q=(8, 8, 8), beta=1.5)),
    ("sph-fp32-band", dict(geometry=wl.SPH, precision="fp32", n_cells=64, Q=(12, 12, 12), beta=1.5)),
    ("sph-fp32-local", dict(geometry=wl.SPH, precision="fp32", n_cells=40, Q=(12, 12, 12), beta=0.0)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_persistent_equals_two_kernels(name, kw):
    d = small_case(**kw)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 31, 0.05)
    used1, f1, m1 = _run(d, f0, True, 7)
    used0, f0b, m0 = _run(d, f0, False, 7)
    assert used1 and not used0
    assert np.array_equal(f1, f0b)
    for k in m1:
        assert np.array_equal(m1[k], m0[k]), k


def test_persistent_with_more_tiles_than_blocks():
    """Two-cell tiles of a 1024-cell cylinder: more tiles than co-resident blocks, so a block
    streams several tiles per stage."""
    d = wl.fourier_cyl_1024()
    P = oracle_problem(d)
    f0 = perturbed_state(P, 5, 0.02)
    used1, f1, _ = _run(d, f0, True, 3, tiling=(2, 0, 0))
    used0, f0b, _ = _run(d, f0, False, 3, tiling=(2, 0, 0))
    assert used1 and not used0
    assert np.array_equal(f1, f0b)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_persistent_matches_oracle(precision):
    d = small_case(geometry=wl.CYL, precision=precision, n_cells=64, Q=(8, 8, 8), beta=1.5, u_wall=(0.1, 0.0))
    P = oracle_problem(d)
    f0 = perturbed_state(P, 12, 0.05)
    used, _, m = _run(d, f0, True, 12)
    assert used
    f_or = osolver.run(f0, P, 12)
    errs = compare_moments(m, osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL[precision], errs


def test_persistent_mass_and_diagnostics():
    """Total mass over many persistent launches (steps split across launches) stays put, and the
    error flag stays clear (every grid barrier completed)."""
    d = small_case(geometry=wl.CYL, precision="fp64", n_cells=48, Q=(8, 8, 8), beta=1.5, u_wall=(0.1, 0.0),
                   T_wall=(1.0, 1.0))
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    assert S.set_persistent_step(True)
    S.set_f(perturbed_state(P, 3, 0.05))
    rc, m0, _, _ = S.diagnostics()
    assert rc == 0
    for k in (1, 2, 5):
        S.step(k)
    rc, m1, _, steps = S.diagnostics()
    assert rc == 0 and steps == 8
    assert abs(m1 - m0) <= 1e-12 * abs(m0)


@pytest.mark.parametrize("persistent", [True, False])
def test_small_tiles_near_the_walls_match_oracle(persistent):
    """400 cells of the 16 x 8 x 8 quadrature: the tile count rounded to the SM count leaves
    tiles of two cells, whose stencils reach the ghost cells of the outer wall from the tile
    before the last.  Five steps against the FP64 oracle."""
    d = dict(wl.fourier_cyl_1024(), n_cells=400)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 17, 0.03)
    S = fdlb.Solver(d)
    used = S.set_persistent_step(persistent)
    assert used == persistent
    S.set_f(f0)
    S.step(5)
    f_or = osolver.run(f0, P, 5)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs
