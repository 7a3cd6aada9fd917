"""Strength of the oracle's pins (CPU).  Each case plants one plausible mistake -- a changed
constant, a dropped factor, a flipped sign, a wrong index or axis -- in a private copy of one
oracle module, built from the module's source text with a single substitution, swaps the copy
into a pin module's namespace, and checks that the pin then fails.  The oracle's own modules are
never modified; the copies live only inside the test."""
import importlib
import inspect
import sys
import types

import pytest

from oracle import geometry as geo
from oracle import solver as osolver

from . import test_oracle_equilibrium as t_eq
from . import test_oracle_geometry as t_geo
from . import test_oracle_kmatrix as t_km
from . import test_oracle_model as t_model
from . import test_oracle_nn as t_nn
from . import test_oracle_quadrature as t_quad
from . import test_oracle_reduced as t_red
from . import test_oracle_solver as t_solver


def planted(monkeypatch, module: str, old: str, new: str):
    """A copy of oracle.<module> with the one occurrence of `old` replaced by `new`, registered
    under a name of its own for the duration of the test (dataclasses look their module up)."""
    real = importlib.import_module(f"oracle.{module}")
    src = inspect.getsource(real)
    assert src.count(old) == 1, (module, old)
    copy = types.ModuleType(f"oracle._planted_{module}")
    copy.__package__ = "oracle"
    copy.__file__ = real.__file__
    monkeypatch.setitem(sys.modules, copy.__name__, copy)
    exec(compile(src.replace(old, new), f"<planted oracle.{module}>", "exec"), copy.__dict__)
    return copy


CYL, SPH = geo.CYL, geo.SPH
LOCAL, FM = osolver.SET_LOCAL, osolver.RET_FM

# (name, module, old, new, pin module, the pin module's name for the oracle module, pin, args)
CASES = [
    # collision term (Eqs. shakhov, j1)
    ("J1 div-u constant", "solver", '(strain + (zeta2 - 2.5) * e(cl["div"])', '(strain + (zeta2 - 1.5) * e(cl["div"])',
     t_solver, "S", "test_collision_momentum_and_energy_moments", (CYL, LOCAL)),
    ("J1 strain factor 2 dropped", "solver", "strain = 2.0 * strain / (2.0 * e(T))", "strain = strain / (2.0 * e(T))",
     t_solver, "S", "test_collision_momentum_and_energy_moments", (CYL, FM)),
    ("J1 Y constant", "solver", 'xi[0] * (e(cl["X"]) + 0.6 * (zeta2 - 2.5) * e(cl["Y"])',
     'xi[0] * (e(cl["X"]) + 0.6 * (zeta2 - 1.5) * e(cl["Y"])',
     t_solver, "S", "test_collision_momentum_and_energy_moments", (CYL, LOCAL)),
    ("J1 X on the second axis", "solver", 'xi[0] * (e(cl["X"])', 'xi[1] * (e(cl["X"])',
     t_solver, "S", "test_collision_momentum_and_energy_moments", (CYL, LOCAL)),
    ("Shakhov xi^2/(5T)", "solver", "fS = fMB * (1.0 + e((1.0 - cl[\"Pr\"]) / (n * T * T)) * (xi2 / (5.0 * e(T)) - 1.0) * xiq)",
     "fS = fMB * (1.0 + e((1.0 - cl[\"Pr\"]) / (n * T * T)) * (xi2 / (3.0 * e(T)) - 1.0) * xiq)",
     t_solver, "S", "test_collision_momentum_and_energy_moments", (SPH, FM)),
    ("sphere strain S_33 dropped", "solver", "S[:, 1, 1] = S[:, 2, 2] = u[:, 0] / R", "S[:, 1, 1] = u[:, 0] / R",
     t_solver, "S", "test_collision_momentum_and_energy_moments", (SPH, LOCAL)),
    # curvature force (Secs. II.B, II.C)
    ("cylinder force sign", "solver", "return kap * (p2 * p2 * KRf - pR * K2f)", "return kap * (p2 * p2 * KRf + pR * K2f)",
     t_solver, "S", "test_force_momentum_and_energy_moments", (CYL, 3)),
    ("sphere force 1/2 dropped", "solver", "return 0.5 * kap * ((p2 * p2 + p3 * p3) * KRf",
     "return kap * ((p2 * p2 + p3 * p3) * KRf", t_solver, "S", "test_force_momentum_and_energy_moments", (SPH, 3)),
    # advection: WENO5, outgoing ghost extrapolation
    ("WENO linear weight", "solver", "a0 = 0.1 / (WENO_EPS + b0) ** 2", "a0 = 0.3 / (WENO_EPS + b0) ** 2",
     t_solver, "S", "test_weno5_flux_difference_converges_at_fifth_order", (1,)),
    ("WENO candidate sign", "solver", "q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0", "q2 = (2.0 * v0 + 5.0 * vp1 + vp2) / 6.0",
     t_solver, "S", "test_weno5_flux_difference_converges_at_fifth_order", (-1,)),
    ("ghost extrapolation coefficient", "solver", "ext[1] = 4 * v[0] - 6 * v[1] + 4 * v[2] - v[3]",
     "ext[1] = 4 * v[0] - 6 * v[1] + 3 * v[2] - v[3]", t_solver, "S", "test_uniform_equilibrium_is_steady", (CYL, 0.0)),
    # diffuse walls (Sec. IV)
    ("wall temperatures swapped", "solver", "Tw, uw = P.T_wall[side], P.u_wall[side]",
     "Tw, uw = P.T_wall[1 - side], P.u_wall[side]", t_solver, "S",
     "test_diffuse_walls_pull_the_adjacent_gas_toward_their_state", (CYL,)),
    ("wall speed dropped", "solver", "g2 = eq.g_full(P.p2, P.w2, P.N2, uw, Tw)",
     "g2 = eq.g_full(P.p2, P.w2, P.N2, 0.0, Tw)", t_solver, "S",
     "test_diffuse_walls_pull_the_adjacent_gas_toward_their_state", (CYL,)),
    # closure gradients
    ("one-sided stencil coefficient", "solver", "d[1] = (-3.0 * phi[0] - 10.0 * phi[1]",
     "d[1] = (-3.0 * phi[0] - 11.0 * phi[1]", t_solver, "S", "test_radial_gradients_converge_at_fourth_order", (1.5,)),
    ("central stencil weight", "solver", "- 8.0 * phi[1:N - 3] + 8.0 * phi[3:N - 1]",
     "- 7.0 * phi[1:N - 3] + 7.0 * phi[3:N - 1]", t_solver, "S", "test_radial_gradients_converge_at_fourth_order", (0.0,)),
    # time integrator
    ("SSP-RK3 stage weight", "solver", "f2 = 0.75 * f + 0.25 * (f1 + dt * rhs(f1, P))",
     "f2 = 0.5 * f + 0.5 * (f1 + dt * rhs(f1, P))", t_solver, "S", "test_ssp_rk3_converges_at_third_order_in_time",
     (CYL, 10)),
    # geometry and Fischer-Methfessel volumes (App. A)
    ("sphere face area R", "geometry", "A_f = R_f ** 2", "A_f = R_f ** 1",
     t_geo, "geo", "test_grid_volumes_and_curvature", (SPH,)),
    ("lens volume coefficient", "geometry", "(dd * dd + 2 * dd * b - 3 * b * b", "(dd * dd + 2 * dd * b - 2 * b * b",
     t_geo, "geo", "test_lens_volume_special_cases", ()),
    ("circle-circle lens term", "geometry", "- 0.5 * np.sqrt(np.maximum(k, 0.0))", "- 0.25 * np.sqrt(np.maximum(k, 0.0))",
     t_geo, "geo", "test_ball_cylinder_volume_matches_appendix_A_formula", (0.3, 1.0, 1.1)),
    # transport model (Sec. II)
    ("Carnahan-Starling power", "model", "(2.0 - eta) / (2.0 * (1.0 - eta) ** 3)", "(2.0 - eta) / (2.0 * (1.0 - eta) ** 2)",
     t_model, "model", "test_chi_matches_carnahan_starling_equation_of_state", ()),
    ("viscosity b rho coefficient", "model", "1.0 / chi + 0.8 * br", "1.0 / chi + 0.6 * br",
     t_model, "model", "test_prandtl_dilute_limit_and_consistency_with_mu_lambda", ()),
    # derivative matrices (Sec. III.B)
    ("K1 factorial", "kmatrix", "K -= np.outer(w * He[l + 1], He[l]) / math.factorial(l)",
     "K -= np.outer(w * He[l + 1], He[l]) / math.factorial(l + 1)", t_km, "km",
     "test_k1_full_differentiates_hermite_gaussians", (4,)),
    ("K2 lower term", "kmatrix", "(l * He[l - 1] if l >= 1 else 0.0)", "((l + 1) * He[l - 1] if l >= 1 else 0.0)",
     t_km, "km", "test_k2_full_differentiates_p_times_hermite_gaussians", (4,)),
    # (the moment identities do not see this one: the jump term's p^0 and p^1 moments vanish by
    # the symmetry of the nodes; exactness on a function continuous at p = 0 does)
    ("half-range jump split", "kmatrix", "jump = np.outer(Phi0, Phi0) / (2.0 * math.sqrt(2.0 * math.pi))",
     "jump = np.outer(Phi0, Phi0) / math.sqrt(2.0 * math.pi)", t_km, "km",
     "test_k_half_exact_on_smooth_polynomial_gaussians", (4,)),
    # equilibrium vectors (Sec. III.C)
    ("full-range equilibrium coefficient", "equilibrium", "2.0 ** s * math.factorial(s) * math.factorial(l - 2 * s)",
     "2.0 ** s * math.factorial(s + 1) * math.factorial(l - 2 * s)", t_eq, "eq",
     "test_full_range_moments_are_gaussian", (8, 7, 0.3, 1.3)),
    ("half-line moment recurrence", "equilibrium", "m[j + 1] = v * m[j] + j * T * m[j - 1]",
     "m[j + 1] = v * m[j] + (j + 1) * T * m[j - 1]", t_eq, "eq", "test_half_range_half_line_moments", (8, 7, 0.3, 1.3)),
    # closure: the gradient of J1's momentum transfer (Eq. j1), seen by the dense-gas momentum balance
    ("J1 gradient without chi", "solver", "X = d_dR(np.log(n * n * chi * T), G)", "X = d_dR(np.log(n * n * T), G)",
     t_solver, "S", "test_dense_fourier_flow_radial_momentum_balance", ()),
    # warm-start network (test infrastructure for the learned warm start)
    ("GELU derivative factor", "nn", "x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)",
     "x * np.exp(-0.5 * x * x) / math.sqrt(math.pi)", t_nn, "nn", "test_gelu_definition", ()),
    ("spectral gradient sign", "nn",
     'g[f"r_im{l}"] = np.einsum("bki,bko->kio", re, dyim) - np.einsum("bki,bko->kio", im, dyre)',
     'g[f"r_im{l}"] = np.einsum("bki,bko->kio", re, dyim) + np.einsum("bki,bko->kio", im, dyre)',
     t_nn, "nn", "test_backward_matches_central_differences", ()),
    ("inverse DFT weight", "nn", "c = np.where(k == 0, 1.0, 2.0)", "c = np.where(k == 0, 2.0, 2.0)",
     t_nn, "nn", "test_dft_pair_matches_numpy_fft", ()),
    ("half-range equilibrium mirror", "equilibrium", "m = half_line_gauss_moments(half * u, T, N)",
     "m = half_line_gauss_moments(u, T, N)", t_eq, "eq", "test_half_range_half_line_moments", (8, 7, 0.3, 1.3)),
    # warm-start seed (Shakhov form of Sec. II) and the steady-state residual
    ("seed Shakhov xi^2/(5T)", "solver", "(xi2 / (5.0 * e(T)) - 1.0) * p[0][None]", "(xi2 / (3.0 * e(T)) - 1.0) * p[0][None]",
     t_solver, "S", "test_shakhov_seed_reproduces_its_moment_profiles", (CYL,)),
    ("seed u_2 dropped from xi^2", "solver", "(p[1][None] - e(u2)) ** 2", "p[1][None] ** 2",
     t_solver, "S", "test_shakhov_seed_reproduces_its_moment_profiles", (SPH,)),
    ("residual without 1/K", "solver", "/ (K * max(float(np.max(np.abs(a))), s))", "/ max(float(np.max(np.abs(a))), s)",
     t_solver, "S", "test_moment_residual_on_a_hand_computed_two_cell_case", ()),
    ("residual scaled by the new profile", "solver", "/ (K * max(float(np.max(np.abs(a))), s))",
     "/ (K * max(float(np.max(np.abs(b))), s))", t_solver, "S", "test_moment_residual_on_a_hand_computed_two_cell_case", ()),
    # reduced cylinder (p_z integrated out)
    ("reduced chi's p_z^2 taken as T", "solver", "(3.0 * T, T))):", "(T, T))):",
     t_red, "S", "test_reduced_collision_is_the_projection", (FM,)),
    ("reduced S2_zz dropped", "solver", "(phi * p2 ** 2).sum(ax), chi.sum(ax),", "(phi * p2 ** 2).sum(ax), zero,",
     t_red, "S", "test_reduced_moments_are_the_projection", ()),
    ("reduced wall mass flux of both members", "solver", "mass = (lambda a: a[..., :1]) if P.reduced else (lambda a: a)",
     "mass = (lambda a: a)", t_red, "S", "test_reduced_mass_conserved_and_seed_carries_its_profiles", ()),
    ("reduced J1 div-u constant", "solver", '(strain_perp + (zeta2 - 2.5) * e(cl["div"])',
     '(strain_perp + (zeta2 - 1.5) * e(cl["div"])', t_red, "S", "test_reduced_collision_is_the_projection", (FM,)),
    ("reduced wall pair without T_w", "solver", "g3 = np.array([1.0, Tw]) if P.reduced", "g3 = np.array([1.0, 1.0]) if P.reduced",
     t_red, "S", "test_reduced_rhs_is_the_projection_under_linear_reconstruction", (LOCAL,)),
    # quadrature (Sec. III.A)
    ("half-range weight formula", "quadrature", "(x + hQ0 ** 2 / math.sqrt(2.0 * math.pi))",
     "(x + hQ0 ** 2 / math.sqrt(math.pi))", t_quad, "quad", "test_half_range_exact_on_half_line_moments", (4,)),
    ("half-range polynomial recurrence", "quadrature", "out[l + 1] = ((x - alpha[l]) * out[l] - b[l] * out[l - 1]) / b[l + 1]",
     "out[l + 1] = ((x - alpha[l]) * out[l] + b[l] * out[l - 1]) / b[l + 1]", t_quad, "quad",
     "test_half_polynomials_orthonormal_and_roots", (5,)),
    ("Hermite Jacobi off-diagonal", "quadrature", "J[n, n - 1] = J[n - 1, n] = math.sqrt(n)",
     "J[n, n - 1] = J[n - 1, n] = math.sqrt(n + 1)", t_quad, "quad", "test_full_range_exact_on_gaussian_moments", (4,)),
]


# pins that run a steady state (tens of seconds): they pass on the oracle in their own module
SLOW_PINS = {"test_dense_fourier_flow_radial_momentum_balance"}


@pytest.mark.parametrize("name,module,old,new,pins,alias,pin,args",
                         [pytest.param(*c, id=c[0], marks=[pytest.mark.slow] if c[6] in SLOW_PINS else [])
                          for c in CASES])
def test_a_planted_mistake_fails_a_pin(monkeypatch, name, module, old, new, pins, alias, pin, args):
    fn = getattr(pins, pin)
    if pin not in SLOW_PINS:
        fn(*args)  # the pin passes on the oracle as it is
    monkeypatch.setattr(pins, alias, planted(monkeypatch, module, old, new))
    with pytest.raises(AssertionError):
        fn(*args)
