"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (largest difference over cells divided by the scale of the quantity):
* FP64 mode: right-hand side and moments <= 1e-10;
* FP32 mode: right-hand side <= 2e-5 of max |L|, moments <= 1e-5 (n / n0, u / sqrt(T0),
  T / T0, q / (n0 T0^1.5)).
"""
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


def _pair(d, seed=11, amp=0.05):
    P = oracle_problem(d)
    f0 = perturbed_state(P, seed, amp)
    S = fdlb.Solver(d)
    S.set_f(f0)
    return P, f0, S


CASES = [
    ("cyl", wl.CYL, 0.0), ("cyl-stretched", wl.CYL, 1.5), ("sph", wl.SPH, 0.0), ("sph-stretched", wl.SPH, 1.2),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,geom,beta", CASES)
def test_rhs_matches_oracle(precision, name, geom, beta):
    d = small_case(geometry=geom, precision=precision, n_cells=37, beta=beta)
    P, f0, S = _pair(d)
    assert S.info()["dt"] == pytest.approx(P.dt, rel=1e-13)
    L_or, det = osolver.rhs(f0, P, details=True)
    L = S.eval_rhs()
    err = np.max(np.abs(L - L_or)) / np.max(np.abs(L_or))
    assert err <= RHS_TOL[precision], err
    cl = S.closure()
    assert np.allclose(cl["nbar"], det["closure"]["nbar"], rtol=1e-12 if precision == "fp64" else 1e-6)
    assert np.allclose(cl["chi"], det["closure"]["chi"], rtol=1e-12 if precision == "fp64" else 1e-6)
    assert np.allclose(cl["tau"], det["closure"]["tau"], rtol=1e-12 if precision == "fp64" else 1e-6)
    assert np.allclose(cl["n_wall"], det["n_wall"], rtol=1e-11 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_moments_of_a_seeded_state(precision):
    d = small_case(precision=precision, n_cells=29)
    P, f0, S = _pair(d, seed=5, amp=0.2)
    errs = compare_moments(S.moments(), osolver.moments(f0, P), P)
    assert max(errs.values()) <= (1e-13 if precision == "fp64" else 2e-7), errs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,geom,beta", CASES)
def test_twenty_steps_match_oracle(precision, name, geom, beta):
    d = small_case(geometry=geom, precision=precision, n_cells=41, beta=beta)
    P, f0, S = _pair(d, seed=3)
    S.step(20)
    f_or = osolver.run(f0, P, 20)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL[precision], errs
    if precision == "fp64":
        assert np.max(np.abs(S.get_f() - f_or)) <= 1e-10 * np.max(np.abs(f_or))


@pytest.mark.parametrize("tiling", [(4, 1, 0), (8, 2, 0), (16, 4, 0), (32, 1, 512), (5, 4, 128), (2, 1, 0), (2, 4, 0)])
def test_tilings_agree(tiling):
    # ragged tails (53 cells), different tile sizes, slice widths and block sizes; tiles of two
    # cells (and one) whose stencils reach ghost cells of a wall they do not touch
    d = small_case(precision="fp64", n_cells=53, u_wall=(0.2, 0.0))
    P, f0, S = _pair(d, seed=9)
    ref = fdlb.Solver(d)
    ref.set_f(f0)
    S.set_tiling(*tiling)
    S.step(7)
    ref.step(7)
    assert np.max(np.abs(S.get_f() - ref.get_f())) <= 1e-13 * np.max(np.abs(f0))


def test_graph_replay_equals_direct_launches():
    d = small_case(precision="fp32", n_cells=30)
    P, f0, S = _pair(d)
    T = fdlb.Solver(d)
    T.set_f(f0)
    S.step(45)  # two graph replays + 5 direct steps
    for _ in range(45):
        T.step(1)
    assert np.array_equal(S.get_f(), T.get_f())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_mass_conservation_on_the_device(precision, geom):
    d = small_case(geometry=geom, precision=precision, n_cells=40, beta=1.0)
    P, f0, S = _pair(d, seed=2)
    _, m0, _, _ = S.diagnostics()
    assert m0 == pytest.approx(osolver.total_mass(f0, P), rel=1e-13 if precision == "fp64" else 1e-7)
    S.step(200)
    rc, m1, _, step = S.diagnostics()
    assert rc == 0 and step == 200
    assert abs(m1 - m0) / m0 <= (1e-12 if precision == "fp64" else 2e-5)


@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_uniform_equilibrium_steady_on_the_device(geom):
    d = small_case(geometry=geom, precision="fp64", n_cells=30, T_wall=(1.0, 1.0), u_wall=(0.0, 0.0),
                   chi_model=fdlb.CHI_SET_LOCAL, beta=1.5)
    S = fdlb.Solver(d)
    f0 = S.get_f()
    S.step(100)
    assert np.max(np.abs(S.get_f() - f0)) <= 1e-12 * np.max(np.abs(f0))


def test_batch_equals_single_instances():
    ds = [small_case(precision="fp32", n_cells=n, Kn=kn, eta0=e, T_wall=(1.0, t), u_wall=(u, 0.0), R=(1.0, r))
          for n, kn, e, t, u, r in ((33, 0.1, 0.2, 1.1, 0.1, 2.0), (64, 0.05, 0.1, 1.3, 0.0, 3.0),
                                    (17, 0.02, 0.25, 1.0, 0.3, 1.5))]
    B = fdlb.Solver(ds)
    B.step(30)
    for q, d in enumerate(ds):
        S = fdlb.Solver(d)
        S.step(30)
        assert np.array_equal(B.get_f(q), S.get_f())


def test_checkpoint_round_trip(tmp_path):
    d = small_case(precision="fp64", n_cells=25)
    P, f0, S = _pair(d)
    S.step(10)
    path = str(tmp_path / "ck.bin")
    S.save(path)
    S.step(10)
    a = S.get_f()
    T = fdlb.Solver(d)
    T.load(path)
    assert T.info()["step"] == 10
    T.step(10)
    assert np.array_equal(a, T.get_f())


def test_error_paths():
    d = small_case(precision="fp64", n_cells=20)
    S = fdlb.Solver(d)
    rc, steps, res = S.run_to_steady(tol=1e-14, max_steps=40, check_every=20)
    assert rc == 4 and steps[0] == 40  # FDLB_ENOTCONVERGED
    with pytest.raises(fdlb.FdlbError):
        S.set_wall(0, 0, -1.0)
    with pytest.raises(fdlb.FdlbError):
        fdlb.Solver(dict(d, Kn=100.0))  # C < 3
    bad = S.get_f()
    bad[3, 1, 1, 1] = np.nan
    S.set_f(bad)
    rc, _, _ = S.run_to_steady(tol=1e-8, max_steps=40, check_every=20)
    assert rc == 6  # FDLB_ENAN


def test_config1_couette_2000_steps_fp64():
    """Cylindrical Couette flow, R 1 -> 2, 64 cells, 8 x 4 x 4 momenta, Kn 0.1, eta0 0.1,
    inner wall speed 0.1, dt 1e-3, FP64, 2000 steps from the uniform equilibrium."""
    d = wl.couette_cyl_64()
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    f_or = osolver.run(osolver.uniform_state(P), P, d["steps"])
    S.step(d["steps"])
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= 1e-10, errs
    assert np.abs(S.moments()["u2"]).max() > 1e-3  # the flow has developed


def test_config2_fourier_cyl_full_size_fp32():
    """Cylindrical Fourier flow at full size: 1024 stretched cells x 1024 momenta, FP32, in the
    launch configuration the benchmark uses; ten steps from a seeded perturbed equilibrium."""
    d = wl.fourier_cyl_1024()
    P, f0, S = _pair(d, seed=21, amp=0.02)
    L = S.eval_rhs()
    L_or = osolver.rhs(f0, P)
    assert np.max(np.abs(L - L_or)) / np.max(np.abs(L_or)) <= RHS_TOL["fp32"]
    S.step(10)
    f_or = osolver.run(f0, P, 10)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs


def test_config3_fourier_sph_full_size_fp32():
    """Spherical Fourier flow at full size: 2048 cells x 3456 momenta (24 x 12 x 12), eta0 0.3,
    seeded Kn; right-hand side and one SSP-RK3 step."""
    from .cases import accept_kn

    d = wl.fourier_sph_2048(accept_kn)
    P, f0, S = _pair(d, seed=22, amp=0.02)
    L = S.eval_rhs()
    L_or = osolver.rhs(f0, P)
    assert np.max(np.abs(L - L_or)) / np.max(np.abs(L_or)) <= RHS_TOL["fp32"]
    S.step(1)
    f_or = osolver.rk3_step(f0, P)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs


def test_batch_instances_of_the_sweep_match_oracle():
    """Three instances of the seeded 512-instance sweep (1024 momenta each, uneven sizes) in one
    batched handle; each compared with the oracle after three steps."""
    from .cases import accept_kn

    ds = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e), n=3)
    S = fdlb.Solver(ds)
    S.step(3)
    for q, d in enumerate(ds):
        P = oracle_problem(d)
        f_or = osolver.run(osolver.uniform_state(P), P, 3)
        errs = compare_moments(S.moments(q), osolver.moments(f_or, P), P)
        assert max(errs.values()) <= TOL["fp32"], (q, errs)


def test_fp32_total_mass_does_not_drift():
    """FP32 populations over 20000 SSP-RK3 steps of a Couette/Fourier instance: the total mass
    sum_c V_c n_c stays within 2e-5 relative.  A stage combination a f_n + b (f + dt L) with
    separately rounded a and b (fl(1/3) + fl(2/3) = 1 + 3e-8) would gain about 3e-4 here."""
    d = small_case(precision="fp32", n_cells=64)
    d.update(Q_R=4, Q_2=4, Q_3=4, u_wall=(0.2, 0.0), T_wall=(1.0, 1.2))
    S = fdlb.Solver(d)
    m0 = S.diagnostics(0)[1]
    S.step(20000)
    m1 = S.diagnostics(0)[1]
    assert abs(m1 - m0) <= 2e-5 * m0, (m0, m1)


def test_programmatic_launch_is_bit_identical():
    """Overlapping kernel prologues with the predecessor (programmatic dependent launch) changes no
    result: 30 steps with and without it, graph-replayed, are equal bit for bit."""
    d = small_case(precision="fp32", n_cells=48)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 9, 0.05)
    out = []
    for on in (True, False):
        S = fdlb.Solver(d)
        S.set_programmatic_launch(on)
        S.set_f(f0)
        S.step(30)
        out.append(S.get_f())
    assert np.array_equal(out[0], out[1])


def test_tensor_core_contraction_matches_oracle():
    """The split-TF32 tensor-core K^h contraction (FP32, 16 x 8 x 8 quadrature at full size): the
    RHS and ten steps against the FP64 oracle within the FP32 tolerances."""
    d = wl.fourier_cyl_1024()
    P, f0, S = _pair(d, seed=21, amp=0.02)
    assert S.set_tensor_contraction(True)
    L = S.eval_rhs()
    L_or = osolver.rhs(f0, P)
    assert np.max(np.abs(L - L_or)) / np.max(np.abs(L_or)) <= RHS_TOL["fp32"]
    S.step(10)
    f_or = osolver.run(f0, P, 10)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs


@pytest.mark.parametrize("threads", [256, 128])
def test_cylinder_fp32_shape_both_vector_widths_match_oracle(threads):
    # the 16 x 8 x 8 cylinder in FP32 has two compile-time kernels: four momenta per thread (blocks
    # of 256) and a whole p_2 row of eight per thread (blocks of at most 128)
    d = small_case(precision="fp32", n_cells=45, Q=(8, 8, 8), u_wall=(0.2, 0.0), T_wall=(1.0, 1.15))
    P, f0, S = _pair(d, seed=4)
    S.set_autotune(0)
    S.set_tiling(6, 8, threads)
    assert S.tiling()["threads"] == threads
    L_or = osolver.rhs(f0, P)
    L = S.eval_rhs()
    assert np.max(np.abs(L - L_or)) / np.max(np.abs(L_or)) <= RHS_TOL["fp32"]
    S.step(20)
    f_or = osolver.run(f0, P, 20)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("slice_k", [1, 2])
def test_sphere_sliced_along_p3_matches_oracle(precision, slice_k):
    # slices narrower than the p_3 axis: K_3 f from its own contraction kernel, the rest of the
    # sphere's stage per slice
    d = small_case(geometry=wl.SPH, precision=precision, n_cells=33, beta=1.2)
    P, f0, S = _pair(d, seed=6)
    S.set_autotune(0)
    S.set_tiling(4, slice_k, 0)
    assert S.tiling()["slice_k"] == slice_k
    L_or = osolver.rhs(f0, P)
    L = S.eval_rhs()
    assert np.max(np.abs(L - L_or)) / np.max(np.abs(L_or)) <= RHS_TOL[precision]
    S.step(20)
    f_or = osolver.run(f0, P, 20)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL[precision], errs
