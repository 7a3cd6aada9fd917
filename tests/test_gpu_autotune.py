"""The autotuner of the tile shapes and the closure's form (fdlb_autotune, automatic tuning at a
batch's first step):
it leaves the state alone, changes no result bit, and its cached choice is reused by a handle of
the same momentum set, precision and size class."""
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
                       Q=(8, 8, 8))
            for n, kn, e, t, u, r in ((133, 0.1, 0.2, 1.1, 0.1, 2.0), (64, 0.05, 0.1, 1.3, 0.0, 3.0),
                                      (217, 0.02, 0.25, 1.0, 0.3, 1.5), (40, 0.3, 0.05, 1.2, 0.2, 4.0))]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tuned_batch_steps_bit_for_bit_like_the_untuned_one(precision):
    ds = _batch(precision)
    A = fdlb.Solver(ds)
    A.set_autotune(0)
    B = fdlb.Solver(ds)  # tunes itself at its first step (a batch)
    A.step(12)
    B.step(12)
    for q in range(len(ds)):
        assert np.array_equal(A.get_f(q), B.get_f(q)), q
    # an explicit re-tune in the middle of the run touches neither the state nor its sums
    f_before = [B.get_f(q) for q in range(len(ds))]
    m_before = [B.moments(q) for q in range(len(ds))]
    B.autotune()
    for q in range(len(ds)):
        assert np.array_equal(B.get_f(q), f_before[q])
        for k, v in B.moments(q).items():
            assert np.array_equal(v, m_before[q][k]), (q, k)
    A.step(13)
    B.step(13)
    for q in range(len(ds)):
        assert np.array_equal(A.get_f(q), B.get_f(q)), q
    assert B.info(0)["step"] == 25


def test_cached_choice_is_reused():
    ds = _batch("fp32")
    A = fdlb.Solver(ds)
    A.autotune()
    t = A.tiling()
    B = fdlb.Solver(ds)
    B.step(1)  # automatic tuning: the cached choice of A's key
    assert B.tiling() == t
    assert 2 <= t["cells_per_tile"] <= 32
    assert (t["closure_form"], t["closure_cells"]) in {("chain", 2), ("chain", 4), ("chain", 8), ("chain", 16),
                                                       ("batch", 28)}


def test_tuned_row_kernel_steps_bit_for_bit_like_the_untuned_one():
    # the 16 x 8 x 8 FP32 cylinder in blocks of 128 threads (a whole p_2 row per thread): the tuner
    # also tries the register bounds of 5, 3 and 2 blocks per SM, which change no result bit
    ds = _batch("fp32")
    A = fdlb.Solver(ds)
    A.set_autotune(0)
    A.set_tiling(0, 0, 128)
    B = fdlb.Solver(ds)
    B.set_autotune(0)
    B.set_tiling(0, 0, 128)
    B.autotune()
    assert A.tiling()["threads"] == 128 and B.tiling()["threads"] == 128
    A.step(12)
    B.step(12)
    for q in range(len(ds)):
        assert np.array_equal(A.get_f(q), B.get_f(q)), q


def test_every_register_bound_of_the_row_kernel_steps_bit_for_bit_alike():
    # the row kernel's variants bounded for 1, 2, 3 and 5 blocks per SM, pinned one by one (tiles of
    # three cells, which five blocks fit): the same populations and moments bit for bit
    ds = _batch("fp32")
    out = {}
    for mb in (1, 2, 3, 5):
        S = fdlb.Solver(ds)
        S.set_autotune(0)
        S.set_tiling(3, 0, 128)
        assert S.stage_min_blocks(mb) == mb
        t = S.tiling()
        assert t["stage_vector_width"] == 8 and t["stage_min_blocks_per_sm"] == mb
        S.step(9)
        out[mb] = ([S.get_f(q) for q in range(len(ds))], S.moments_all())
    for mb in (2, 3, 5):
        for q in range(len(ds)):
            assert np.array_equal(out[mb][0][q], out[1][0][q]), (mb, q)
        assert np.array_equal(out[mb][1], out[1][1]), mb


def test_a_register_bound_not_built_for_the_shape_is_refused():
    S = fdlb.Solver(_batch("fp32"))
    S.set_autotune(0)
    S.set_tiling(3, 0, 128)
    before = S.tiling()
    with pytest.raises(fdlb.FdlbError):
        S.stage_min_blocks(4)
    assert S.tiling() == before
    D = fdlb.Solver(_batch("fp64"))
    D.set_autotune(0)
    with pytest.raises(fdlb.FdlbError):
        D.stage_min_blocks(5)
    assert D.stage_min_blocks(1) == 1
