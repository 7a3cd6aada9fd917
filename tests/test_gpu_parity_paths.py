"""Parity with the FP64 oracle of the paths around the step: the steady-state residual the
library reports, the warm-start seed (from moment profiles and from the network), a dense gas at
rest with the Fischer-Methfessel chi, more steps at the full spherical size, and sixteen
instances of the seeded sweep in one batched handle.

The oracle runs of the sweep instances go to a process pool started with the spawn method (a
pool forked after the first GPU call would inherit the CUDA context)."""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

from oracle import nn as onn
from oracle import solver as osolver
from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import warmstart as ws
from paper_2403_15051_gb300 import workloads as wl

from .cases import accept_kn, compare_moments, oracle_problem, perturbed_state, small_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _scales(P):
    T0 = 0.5 * (P.T_wall[0] + P.T_wall[1])
    return (P.n0, 1.0, T0, P.n0 * T0 ** 1.5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_reported_residual_matches_oracle(precision, geom):
    """fdlb_run_to_steady's residual after one check interval of K steps against the oracle's
    moment_residual of the profiles before and after the same K steps (FP64 moments in both)."""
    K = 20
    d = small_case(geometry=geom, precision=precision, n_cells=37, beta=1.0)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 13, 0.05)
    S = fdlb.Solver(d)
    S.set_f(f0)
    rc, steps, res = S.run_to_steady(tol=1e-300, max_steps=K, check_every=K)
    assert rc == 4 and steps[0] == K  # FDLB_ENOTCONVERGED after the one interval
    r_or = osolver.moment_residual(osolver.profile_moments(f0, P), osolver.profile_moments(osolver.run(f0, P, K), P),
                                   K, _scales(P))
    assert r_or > 1e-6
    # FP32: the moments after K steps agree to ~1e-6 of their scales, the K-step change is ~1e-2
    assert res[0] == pytest.approx(r_or, rel=1e-9 if precision == "fp64" else 2e-3)
    # the last residual is also what fdlb_get_diagnostics reports
    assert S.diagnostics()[2] == res[0]


def _seed_profiles(P, n_points):
    xp = np.linspace(0.0, 1.0, n_points)
    n = P.n0 * (1.0 + 0.15 * np.sin(3.0 * xp))
    u2 = 0.2 * np.cos(2.0 * xp) if P.geometry == wl.CYL else 0.0 * xp
    T = 1.0 + 0.2 * xp * xp
    qR = 0.02 * P.n0 * np.cos(5.0 * xp)
    return xp, n, u2, T, qR


def _on_cells(P, xp, prof):
    G = P.grid
    xc = (G.R_c - G.R_f[0]) / (G.R_f[-1] - G.R_f[0])
    return [np.interp(xc, xp, v) for v in prof]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_init_from_moments_matches_oracle_seed(precision, geom):
    """fdlb_init_from_moments (profiles at 33 points of the normalised radius, linear
    interpolation onto the cells) against the oracle's shakhov_seed of the same cell profiles,
    element by element."""
    d = small_case(geometry=geom, precision=precision, n_cells=45, Q=(5, 4, 6), beta=1.2)
    P = oracle_problem(d)
    xp, *prof = _seed_profiles(P, 33)
    S = fdlb.Solver(d)
    S.init_from_moments(0, *prof)
    f = S.get_f()
    f_or = osolver.shakhov_seed(P, *_on_cells(P, xp, prof))
    err = np.max(np.abs(f - f_or)) / np.max(np.abs(f_or))
    assert err <= (1e-12 if precision == "fp64" else 1e-6), err
    assert S.info()["step"] == 0


def test_network_warm_start_matches_oracle():
    """fdlb_nn_warm_start end to end: the network's profiles (the FP64 oracle network with the same
    BF16 weights), decoded as the header states (n = n0 (1 + o0), u_2 = 0.1 o1,
    T = T_in (1 + 0.1 o2), q_R = 0.01 n0 T_in^1.5 o3), n and q_R scaled together so that the seed
    carries the mass of the instance's uniform start, then the Shakhov seed on the cells."""
    from .test_gpu_nn import bf16_round, normalise

    sizes = dict(W=32, m=6, L=2, H=64, P=96)
    theta = bf16_round(onn.init_params(7, W=sizes["W"], m=sizes["m"], L=sizes["L"], H=sizes["H"]))
    rng = np.random.default_rng(3)
    lay, _ = onn.layout(sizes["W"], sizes["m"], sizes["L"], sizes["H"])
    for k, (o, s) in lay.items():  # biases and spectral weights large enough to shape the profiles
        n = int(np.prod(s))
        if k.startswith("r_"):
            theta[o:o + n] = bf16_round(rng.normal(0, 0.5 / sizes["W"], n))
        if k.endswith("_b") or (k[0] == "b" and k[1:].isdigit()):
            theta[o:o + n] = bf16_round(rng.normal(0, 0.1, n))
    net = fdlb.WarmStartNet(sizes["W"], sizes["m"], sizes["L"], sizes["H"], sizes["P"], max_batch=4)
    net.set_params(theta.astype(np.float32))
    d = small_case(precision="fp64", n_cells=40, Kn=0.08, eta0=0.15, T_wall=(1.0, 1.2), u_wall=(0.2, 0.0),
                   R=(1.0, 2.5))
    raw = ws.raw_parameters(d)
    S = fdlb.Solver(d)
    net.warm_start(S, 0, raw)
    f = S.get_f()
    P = oracle_problem(d)
    out, _ = onn.forward(theta, normalise(raw[None].astype(np.float64)), P=sizes["P"], W=sizes["W"], m=sizes["m"],
                         L=sizes["L"], H=sizes["H"])
    o = out[0]
    xp = np.linspace(0.0, 1.0, sizes["P"])
    prof = [P.n0 * np.maximum(0.05, 1.0 + o[:, 0]), 0.1 * o[:, 1], np.maximum(0.05, 1.0 + 0.1 * o[:, 2]),
            0.01 * P.n0 * o[:, 3]]
    seed = osolver.shakhov_seed(P, *_on_cells(P, xp, prof))
    lam = osolver.total_mass(osolver.uniform_state(P), P) / osolver.total_mass(seed, P)
    prof[0] = prof[0] * lam
    prof[3] = prof[3] * lam
    f_or = osolver.shakhov_seed(P, *_on_cells(P, xp, prof))
    assert abs(lam - 1.0) > 1e-4  # the rescaling is exercised
    # the network's FP32 activations against FP64: outputs agree to ~1e-4
    assert np.max(np.abs(f - f_or)) <= 2e-3 * np.max(np.abs(f_or))
    assert S.diagnostics()[1] == pytest.approx(osolver.total_mass(osolver.uniform_state(P), P), rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_dense_gas_at_rest_twenty_steps_match_oracle(precision, geom):
    """The gas-at-rest instance eta0 = 0.2, R_L = 1, C = 4 (sigma = 1, 96 cells, Fischer-Methfessel
    chi over a 24-cell band): twenty steps from the uniform start against the oracle."""
    d = [x for x in wl.layering_instances(geom, precision=precision)
         if x["eta0"] == 0.2 and x["R_in"] == 1.0 and x["R_out"] == 5.0][0]
    P = oracle_problem(d)
    S = fdlb.Solver(d)
    S.step(20)
    f_or = osolver.run(osolver.uniform_state(P), P, 20)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL[precision], errs
    cl = S.closure()
    _, det = osolver.rhs(f_or, P, details=True)
    assert np.allclose(cl["nbar"], det["closure"]["nbar"], rtol=1e-11 if precision == "fp64" else 1e-5)
    # the layering has started: the density next to the walls has moved off n0
    assert np.max(np.abs(S.moments()["n"] / P.n0 - 1.0)) > 1e-4


@pytest.mark.slow
def test_config3_fourier_sph_full_size_five_steps_fp32():
    """Spherical Fourier flow at full size (2048 cells x 3456 momenta, eta0 0.3, seeded Kn): five
    SSP-RK3 steps from a seeded perturbed equilibrium against the oracle."""
    d = wl.fourier_sph_2048(accept_kn)
    P = oracle_problem(d)
    f0 = perturbed_state(P, 23, 0.02)
    S = fdlb.Solver(d)
    S.set_f(f0)
    S.step(5)
    f_or = osolver.run(f0, P, 5)
    errs = compare_moments(S.moments(), osolver.moments(f_or, P), P)
    assert max(errs.values()) <= TOL["fp32"], errs


def _oracle_moments_after(d, steps):
    P = oracle_problem(d)
    return osolver.moments(osolver.run(osolver.uniform_state(P), P, steps), P)


@pytest.mark.slow
def test_sixteen_sweep_instances_match_oracle():
    """Sixteen instances of the seeded 512-instance sweep (1024 momenta each, 133 to 1762 cells) in
    one batched handle, three steps, each against the oracle."""
    ds = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e), n=16)
    S = fdlb.Solver(ds)
    S.step(3)
    got = [S.moments(q) for q in range(len(ds))]
    S.close()
    with cf.ProcessPoolExecutor(max_workers=8, mp_context=mp.get_context("spawn")) as ex:
        ref = list(ex.map(_oracle_moments_after, ds, [3] * len(ds)))
    for q, d in enumerate(ds):
        errs = compare_moments(got[q], ref[q], oracle_problem(d))
        assert max(errs.values()) <= TOL["fp32"], (q, errs)
