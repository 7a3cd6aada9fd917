"""The C-ABI library on the CPU: it loads, exports every symbol the header declares, its host
set-up (quadrature, derivative matrices, grid, FM weights, parameters) matches the oracle, and
the device entry points fail loudly without a GPU."""
import os
import re

import numpy as np
import pytest

from oracle import geometry as ogeo
from oracle import kmatrix as okm
from oracle import model as omodel
from oracle import quadrature as oquad
from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb

from .cases import ROOT, oracle_problem, small_case


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fdlb.load_library()


def test_every_declared_symbol_is_exported(lib):
    header = open(os.path.join(ROOT, "include", "fdlb.h")).read()
    names = sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char\*)\s+(fdlb_\w+)\s*\(", header, re.M)))
    assert len(names) >= 28
    for n in names:
        assert hasattr(lib, n), n


def test_library_leaves_no_symbol_of_its_own_unresolved(lib):
    # every undefined symbol of the shared library is a versioned one of the system libraries (an
    # internal function declared with the wrong linkage would show here, unversioned)
    import shutil
    import subprocess

    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    so = os.path.join(ROOT, "paper_2403_15051_gb300", "libfdlb_gb300.so")
    out = subprocess.run([nm, "-D", "--undefined-only", so], capture_output=True, text=True, check=True).stdout
    own = [ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-2:-1] == ["U"] and "@" not in ln]
    assert own == [], own


@pytest.mark.parametrize("Q", [1, 2, 4, 8, 12, 16, 24, 40, 60, 100])
def test_quadrature_matches_oracle(lib, Q):
    x, w = fdlb.quadrature(fdlb.QUAD_HALF, Q)
    xo, wo = oquad.half_range_axis(Q)
    assert np.allclose(x, xo, rtol=0, atol=1e-13 * max(1.0, np.abs(xo).max()))
    assert np.allclose(w, wo, rtol=1e-12)
    if Q > 24:  # the full-range axes stop at order 24
        return
    x, w = fdlb.quadrature(fdlb.QUAD_FULL, Q)
    xo, wo = oquad.full_range_rule(Q)
    assert np.allclose(x, xo, atol=1e-13 * max(1.0, np.abs(xo).max()))
    assert np.allclose(w, wo, rtol=1e-12)


@pytest.mark.parametrize("Q", [1, 2, 4, 8, 12, 24, 40, 100])
def test_derivative_matrices_match_oracle(lib, Q):
    K = fdlb.derivative_matrix(fdlb.QUAD_HALF, Q)
    x, lam, a, b = oquad.half_range_rule(Q)
    p, w = np.concatenate([x, -x]), np.concatenate([lam, lam])
    Ko = okm.k1_half(p, w, a, b)
    assert np.allclose(K * w[None, :], Ko * w[None, :], atol=1e-13 * max(1.0, np.abs(Ko * w[None, :]).max()))
    if Q > 24:  # the full-range axes stop at order 24
        return
    K2 = fdlb.derivative_matrix(fdlb.QUAD_FULL, Q)
    xf, wf = oquad.full_range_rule(Q)
    K2o = okm.k2_full(xf, wf)
    assert np.allclose(K2 * wf[None, :], K2o * wf[None, :], atol=1e-13 * max(1.0, np.abs(K2o * wf).max()))


def test_physical_parameters_match_oracle_and_table_I(lib):
    for C, eta0 in ((4, 0.01), (7, 0.1), (10, 0.2)):
        kn = omodel.knudsen(C, eta0)
        Cl, s, n0 = fdlb.physical_parameters(kn, eta0, 2.0)
        Co, so, n0o = omodel.physical_parameters(kn, eta0, 2.0)
        assert Cl == pytest.approx(C, rel=1e-13) and s == pytest.approx(so, rel=1e-13) and n0 == pytest.approx(n0o, rel=1e-13)


@pytest.mark.parametrize("g", [0, 1])
@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_grid_and_fm_weights_match_oracle(lib, g, beta):
    sigma, N = 0.22, 48
    Rc, Rf, V, kap = fdlb.grid(g, 1.0, 2.7, sigma, N, beta)
    G = ogeo.make_grid(g, 1.0, 2.7, sigma, N, beta)
    for a, b in ((Rc, G.R_c), (Rf, G.R_f), (V, G.V_c), (kap, G.kappa)):
        # thin shells: (b^3 - a^3)/3 cancels, so allow a few ulps of the difference
        assert np.allclose(a, b, rtol=1e-12, atol=1e-15)
    W = fdlb.fm_weights(g, 1.0, 2.7, sigma, N, beta)
    Wo = ogeo.fm_weights(G, sigma)
    assert np.max(np.abs(W - Wo)) < 1e-12


def test_workspace_size_is_host_logic_and_rejects_bad_parameters(lib):
    import ctypes
    d = small_case()
    p = (fdlb.Params * 1)(fdlb.make_params(d))
    nb = ctypes.c_size_t()
    assert lib.fdlb_workspace_bytes(p, 1, ctypes.byref(nb)) == 0 and nb.value > 0
    for bad in (dict(n_cells=4), dict(Q_R=0), dict(eta0=0.7), dict(T_wall=(-1.0, 1.0)), dict(Kn=50.0)):
        q = dict(d)
        q.update(bad)
        pp = (fdlb.Params * 1)(fdlb.make_params(q))
        assert lib.fdlb_workspace_bytes(pp, 1, ctypes.byref(nb)) == 1  # FDLB_EINVAL
    # N >= Q is rejected
    q = dict(d, N_R=4)
    pp = (fdlb.Params * 1)(fdlb.make_params(q))
    assert lib.fdlb_workspace_bytes(pp, 1, ctypes.byref(nb)) == 1


def test_create_fails_loudly_without_a_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fdlb.FdlbError):
        fdlb.Solver(small_case(), use_torch_workspace=False)


def test_default_time_step_matches_oracle_rule(lib):
    # the CFL / relaxation-time rule is host logic; compare through the workspace-free plan:
    # dt of the oracle problem against the formula restated here from the same inputs
    d = small_case(dt=None)
    P = oracle_problem(d)
    dr = np.min(np.diff(P.grid.R_f))
    chi0 = float(omodel.chi_set(d["eta0"]))
    tau = float(omodel.relaxation_time(P.n0, 1.2, chi0, P.sigma))
    assert P.dt == pytest.approx(min(0.4 * dr / (np.abs(P.pR).max() * np.sqrt(1.2)), 0.5 * tau), rel=1e-14)


@pytest.mark.parametrize("maker", ["layering", "heatflux"])
@pytest.mark.parametrize("geometry", [0, 1])
def test_sweep_workloads_pass_host_validation(lib, maker, geometry):
    """The gas-at-rest and heat-flux sweeps are valid batches for the library's set-up."""
    import ctypes

    from paper_2403_15051_gb300 import workloads as wl
    ds = (wl.layering_instances if maker == "layering" else wl.heatflux_instances)(geometry)
    p = (fdlb.Params * len(ds))(*[fdlb.make_params(d) for d in ds])
    nb = ctypes.c_size_t()
    assert lib.fdlb_workspace_bytes(p, len(ds), ctypes.byref(nb)) == 0 and nb.value > 0


def test_handle_calls_reject_a_null_handle(lib):
    import ctypes
    null = ctypes.c_void_p(0)
    d, n1, n2 = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    used = ctypes.c_int()
    assert lib.fdlb_set_persistent_step(null, 1, ctypes.byref(used)) == 1
    assert lib.fdlb_set_wait_test(null, 0, 0) == 1
    assert lib.fdlb_clear_error(null) == 1
    assert lib.fdlb_step_kernel_times(null, ctypes.byref(d), ctypes.byref(n1), ctypes.byref(n2)) == 1
    assert lib.fdlb_set_stage_min_blocks(null, 1, ctypes.byref(used)) == 1
    assert lib.fdlb_set_closure_form(null, 0, ctypes.byref(used)) == 1


def test_params_marshalling_rejects_an_unknown_precision():
    d = small_case()
    assert fdlb.make_params(dict(d, precision="fp32")).precision == fdlb.FP32
    assert fdlb.make_params(dict(d, precision="fp64")).precision == fdlb.FP64
    for bad in ("bf16", "f32", "FP32", 2):
        with pytest.raises(ValueError):
            fdlb.make_params(dict(d, precision=bad))
        with pytest.raises(ValueError):  # raised before any device pointer is used
            fdlb.moments_noalloc(bad, 2, 2, 2, 16, 0, 0)


def test_fm_band_beyond_32_bit_offsets_is_rejected_before_allocation(lib):
    """65536 cells across a gap of three diameters: every ball reaches two thirds of the cells, so
    the Fischer-Methfessel band would hold 2.9e9 entries (23 GB), more than the device tables'
    32-bit offsets address.  The set-up refuses it with FDLB_EINVAL before allocating; with the
    local chi (no band) the same grid plans normally."""
    import ctypes
    nb = ctypes.c_size_t()
    base = dict(small_case(), R_in=1.0, R_out=4.0, n_cells=65536, sigma=1.0, Kn=None, Q_R=2, Q_2=2, Q_3=2)
    p = (fdlb.Params * 1)(fdlb.make_params(dict(base, chi_model=fdlb.CHI_RET_FM)))
    assert lib.fdlb_workspace_bytes(p, 1, ctypes.byref(nb)) == 1  # FDLB_EINVAL
    p = (fdlb.Params * 1)(fdlb.make_params(dict(base, chi_model=fdlb.CHI_SET_LOCAL)))
    assert lib.fdlb_workspace_bytes(p, 1, ctypes.byref(nb)) == 0 and nb.value > 0


def test_reduced_cylinder_parameters(lib):
    """FDLB_CYL_Z (p_z integrated out) takes Q_3 = 0 and plans a state of 2 x 2Q_R x Q_2 populations
    per cell; a third-axis order is refused."""
    import ctypes

    from paper_2403_15051_gb300 import workloads as wl

    d = wl.couette_cyl_reduced(Q_R=6, Q_2=4)
    nb = ctypes.c_size_t()
    arr = (fdlb.Params * 1)(fdlb.make_params(d))
    assert lib.fdlb_workspace_bytes(arr, 1, ctypes.byref(nb)) == 0 and nb.value > 3 * d["n_cells"] * 2 * 12 * 4 * 4
    arr = (fdlb.Params * 1)(fdlb.make_params(dict(d, Q_3=4)))
    assert lib.fdlb_workspace_bytes(arr, 1, ctypes.byref(nb)) == 1  # FDLB_EINVAL
