"""Pins of the oracle's reduced cylinder (p_z integrated out; Sec. III.A's remark on the trivial axes
of Couette flow).  The reduced pair of a full-model state that is even in p_z is
phi = sum_k f_k, chi = sum_k p_k^2 f_k over the p_z nodes; the moments, the curvature force and the
collision of the reduced model must be those projections of the full model's, to round-off, as
long as the full model's discrete p_z equilibrium reproduces the Gaussian moments the collision
needs (int g = 1, int p^2 g = T, int p^4 g = 3 T^2: expansion order N_3 >= 4).  The advection
(WENO5 on each member) is not a projection of the full one (the weights are nonlinear), so the
reduced run is pinned by exact mass conservation, the steady uniform equilibrium, and its agreement
with the full model at steady state."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import solver as S
from paper_2403_15051_gb300 import workloads as wl


def _pair(Q3=8, n_cells=20, **kw):
    args = dict(eta0=0.15, Kn=0.08, T_wall=(1.0, 1.2), u_wall=(0.2, 0.0), beta=0.7)
    args.update(kw)
    full = S.make_problem(geo.CYL, 1.0, 2.5, n_cells, 5, 6, Q3, **args)
    red = S.make_problem(geo.CYL, 1.0, 2.5, n_cells, 5, 6, 0, reduced=True, **args)
    return full, red


def _even_state(P, seed=4, amp=0.1):
    f = S.uniform_state(P) * wl.perturbation(P.shape, seed, amp)
    return 0.5 * (f + f[..., ::-1])  # the p_z nodes are symmetric: f even in p_z


def _project(f, P):
    return np.stack([f.sum(-1), (f * P.p3[None, None, None, :] ** 2).sum(-1)], axis=-1)


def test_reduced_moments_are_the_projection():
    full, red = _pair()
    f = _even_state(full)
    Sf, Sr = S.raw_sums(f, full), S.raw_sums(_project(f, full), red)
    # per sum, relative to its own size; the odd p_z sums are zero up to the full model's rounding
    scale = np.maximum(np.abs(Sf).max(0), 0.1 * np.abs(Sf[:, 0]).max())
    assert np.all(np.abs(Sf - Sr) <= 1e-13 * scale)


def test_reduced_force_is_the_projection():
    full, red = _pair()
    f = _even_state(full)
    a, b = _project(S.force(f, full), full), S.force(_project(f, full), red)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("chi_model", [S.RET_FM, S.SET_LOCAL])
def test_reduced_collision_is_the_projection(chi_model):
    full, red = _pair(chi_model=chi_model)
    f = _even_state(full)
    clf = S.closure(f, full)
    clr = S.closure(_project(f, full), red)
    for k in ("n", "T", "tau", "Pr", "X", "Y", "div"):
        assert np.allclose(clf[k], clr[k], rtol=1e-12, atol=1e-14), k
    a = _project(S.collision(f, full, clf), full)
    b = S.collision_reduced(_project(f, full), red, clr)
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))


def test_projection_needs_the_fourth_moment_of_the_p_z_equilibrium():
    # with Q_3 = 4 the expansion stops at N_3 = 3, so sum g p^4 misses 3 (T - 1)^2 and chi's
    # collision differs from the reduced one (the pin above is not vacuous)
    full, red = _pair(Q3=4, T_wall=(1.0, 1.6))
    f = _even_state(full, amp=0.2)
    a = _project(S.collision(f, full, S.closure(f, full)), full)
    b = S.collision_reduced(_project(f, full), red, S.closure(_project(f, full), red))
    assert np.max(np.abs(a[..., 1] - b[..., 1])) > 1e-6 * np.max(np.abs(a[..., 1]))


def test_reduced_mass_conserved_and_seed_carries_its_profiles():
    _, red = _pair(n_cells=24)
    f = S.uniform_state(red) * wl.perturbation(red.shape, 6, 0.05)
    m0 = S.total_mass(f, red)
    f = S.run(f, red, 20)
    assert abs(S.total_mass(f, red) - m0) / m0 < 1e-13
    # the seed carries q_R exactly once the expansions reach degree 6 in p_R and 4 in p_2 (as in
    # the full model): Q_R = 8, Q_2 = 6
    red = S.make_problem(geo.CYL, 1.0, 2.5, 24, 8, 6, 0, reduced=True, eta0=0.15, Kn=0.08)
    x = (np.arange(24) + 0.5) / 24
    n, u2, T, qR = red.n0 * (1 + 0.1 * x), 0.2 * x, 1.0 + 0.2 * x, 0.02 * red.n0 * np.cos(x)
    m = S.moments(S.shakhov_seed(red, n, u2, T, qR), red)
    assert np.allclose(m["n"], n, rtol=1e-13) and np.allclose(m["T"], T, rtol=1e-12)
    assert np.max(np.abs(m["u"][:, 1] - u2)) < 1e-13 and np.max(np.abs(m["q"][:, 0] - qR)) < 1e-12 * red.n0


def test_reduced_uniform_equilibrium_is_steady():
    _, red = _pair(T_wall=(1.0, 1.0), u_wall=(0.0, 0.0), chi_model=S.SET_LOCAL)
    f = S.uniform_state(red, T0=1.0)
    g = S.run(f, red, 5)
    assert np.max(np.abs(g - f)) <= 1e-13 * np.max(np.abs(f))


@pytest.mark.parametrize("chi_model", [S.RET_FM, S.SET_LOCAL])
def test_reduced_rhs_is_the_projection_under_linear_reconstruction(chi_model):
    """With the WENO weights pinned to their linear values (epsilon far above every smoothness
    indicator) the reconstruction is linear, so the whole right-hand side, walls and ghost cells
    included, projects exactly: the reduced L of the projected state is the projected full L."""
    full, red = _pair(chi_model=chi_model)
    f = _even_state(full)
    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(S, "WENO_EPS", 1e12)
        a = _project(S.rhs(f, full), full)
        b = S.rhs(_project(f, full), red)
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(a))


@pytest.mark.slow
def test_reduced_and_full_runs_agree():
    """A thousand steps of Couette/Fourier flow between cylinders from the uniform start: the reduced
    and the full model (N_3 = 7) differ only through the advection's nonlinear WENO weights, at the
    1e-3 level of the moments."""
    full, red = _pair(n_cells=16, Q3=8)
    steps = int(round(6.0 / full.dt))
    mf = S.moments(S.run(S.uniform_state(full), full, steps), full)
    mr = S.moments(S.run(S.uniform_state(red), red, steps), red)
    assert np.max(np.abs(mf["n"] - mr["n"])) < 1e-3 * full.n0
    assert np.max(np.abs(mf["u"][:, 1] - mr["u"][:, 1])) < 1e-3
    assert np.max(np.abs(mf["T"] - mr["T"])) < 1e-3
