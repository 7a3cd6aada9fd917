"""Workload definitions and seeded synthetic inputs shared by the tests, the benchmark and
the oracle-side checks.

This module holds sizes, physical parameters and random numbers only - none of the
method's arithmetic.  Both the CUDA path and the oracle receive what it returns as plain
numbers and compute everything else with their own code.

Workloads (the paper's three flow set-ups of Sec. IV at sizes chosen for this library):

* ``couette_cyl_64``   cylindrical Couette flow, R 1 -> 2, 64 uniform cells, half-range order 4 on
  p_R x full-range order 4 on p_phi and p_z (128 momenta), Kn 0.1, eta0 0.1, inner wall speed
  0.1, T_w = 1, dt 1e-3, FP64, 2000 SSP-RK3 steps from the uniform equilibrium;
* ``fourier_cyl_1024`` cylindrical Fourier flow, R 1 -> 3, 1024 tanh-stretched cells (beta 1.5),
  16 x 8 x 8 = 1024 momenta, Kn 0.05, eta0 0.2, T 1.0 / 1.1, walls at rest, FP32 populations;
* ``fourier_sph_2048`` spherical Fourier flow, r 1 -> 4, 2048 uniform cells, 24 x 12 x 12 = 3456
  momenta, eta0 0.3, T 1.0 / 1.2, Kn drawn log-uniform in [0.01, 1] from seed 0 and redrawn
  until the caller's acceptance test (confinement C >= 3) holds, FP32 populations;
* ``batch_512``        512 cylindrical Couette/Fourier instances with 1024 momenta each, radial size
  uniform in [128, 2048], Kn log-uniform in [0.01, 1], eta0 uniform in [0.01, 0.3], radius ratio
  uniform in [1.2, 5], inner wall speed uniform in [0, 0.3], outer/inner wall temperature ratio
  uniform in [1.0, 1.3], from one seed, redrawn under the same acceptance test.
"""
from __future__ import annotations

import numpy as np

CYL = 0
SPH = 1
CYL_Z = 2  # cylinder with p_z integrated out: the pair (phi, chi) in place of the p_z nodes


def couette_cyl_64():
    return dict(geometry=CYL, R_in=1.0, R_out=2.0, n_cells=64, beta=0.0, Q_R=4, Q_2=4, Q_3=4,
                Kn=0.1, eta0=0.1, T_wall=(1.0, 1.0), u_wall=(0.1, 0.0), dt=1e-3, precision="fp64",
                steps=2000)


def fourier_cyl_1024():
    return dict(geometry=CYL, R_in=1.0, R_out=3.0, n_cells=1024, beta=1.5, Q_R=8, Q_2=8, Q_3=8,
                Kn=0.05, eta0=0.2, T_wall=(1.0, 1.1), u_wall=(0.0, 0.0), dt=None, precision="fp32")


def couette_cyl_reduced(Q_R=20, Q_2=8, eta0=0.1, C=4.0, R_L=1.0, cells_per_sigma=24, precision="fp32"):
    """Cylindrical Couette flow on the paper's HHLB(7, Q_R) x HLB(7, 8) quadrature with p_z integrated
    out (Sec. IV.A): sigma = 1, inner radius R_L, outer R_L + C, inner wall moving at U_w = sqrt(T_w),
    T_w = 1 on both walls."""
    return dict(geometry=CYL_Z, R_in=R_L, R_out=R_L + C, sigma=1.0, n_cells=int(round(C * cells_per_sigma)), beta=0.0,
                Q_R=Q_R, Q_2=Q_2, Q_3=0, eta0=eta0, T_wall=(1.0, 1.0), u_wall=(1.0, 0.0), dt=None,
                precision=precision, chi_model=0)


def draw_log_uniform_kn(rng, accept, lo=0.01, hi=1.0, max_draws=10_000):
    """Kn = 10^U[log10 lo, log10 hi], redrawn until accept(Kn) is true."""
    for _ in range(max_draws):
        kn = float(10.0 ** rng.uniform(np.log10(lo), np.log10(hi)))
        if accept(kn):
            return kn
    raise RuntimeError("no accepted draw")


def fourier_sph_2048(accept_kn):
    """accept_kn(Kn, eta0) -> bool is supplied by the caller (the C >= 3 test)."""
    rng = np.random.default_rng(0)
    eta0 = 0.3
    kn = draw_log_uniform_kn(rng, lambda k: accept_kn(k, eta0))
    return dict(geometry=SPH, R_in=1.0, R_out=4.0, n_cells=2048, beta=0.0, Q_R=12, Q_2=12, Q_3=12,
                Kn=kn, eta0=eta0, T_wall=(1.0, 1.2), u_wall=(0.0, 0.0), dt=None, precision="fp32")


def batch_instances(accept, n=512, seed=0, n_lo=128, n_hi=2048):
    """Parameter-sweep instances (cylindrical, 1024 momenta).  accept(Kn, eta0, R_out) -> bool."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        n_cells = int(rng.integers(n_lo, n_hi + 1))
        kn = float(10.0 ** rng.uniform(-2.0, 0.0))
        eta0 = float(rng.uniform(0.01, 0.3))
        ratio = float(rng.uniform(1.2, 5.0))
        uw = float(rng.uniform(0.0, 0.3))
        tr = float(rng.uniform(1.0, 1.3))
        if not accept(kn, eta0, ratio):
            continue
        out.append(dict(geometry=CYL, R_in=1.0, R_out=ratio, n_cells=n_cells, beta=0.0, Q_R=8, Q_2=8,
                        Q_3=8, Kn=kn, eta0=eta0, T_wall=(1.0, tr), u_wall=(uw, 0.0), dt=None,
                        precision="fp32"))
    return out


def layering_instances(geometry, precision="fp32", cells_per_sigma=24, Q=(4, 4, 4), etas=(0.01, 0.1, 0.2),
                       radii=(1.0, 3.0, 5.0), confinements=(4.0, 7.0, 10.0)):
    """Dense hard-sphere gas at rest between coaxial cylinders or concentric spheres at T_w = 1 (the
    appendix on the stationary gas): sigma = 1, inner radius R_L, outer R_L + C, mean reduced density
    eta0; every combination, in the order eta0, R_L, C."""
    out = []
    for eta0 in etas:
        for rl in radii:
            for c in confinements:
                out.append(dict(geometry=geometry, R_in=rl, R_out=rl + c, sigma=1.0, n_cells=int(round(c * cells_per_sigma)),
                                beta=0.0, Q_R=Q[0], Q_2=Q[1], Q_3=Q[2], eta0=eta0, T_wall=(1.0, 1.0), u_wall=(0.0, 0.0),
                                dt=None, precision=precision, chi_model=0))
    return out


def heatflux_instances(geometry, precision="fp64", cells_per_sigma=24, Q=(4, 4, 4), etas=(0.01, 0.1, 0.2),
                       radii=(1.0, 2.0, 5.0, 10.0, 20.0, 50.0), confinement=4.0, dT=0.1):
    """Fourier flow between coaxial cylinders or concentric spheres at rest with wall temperatures
    1 and 1 + dT (the comparison of the two geometries' heat fluxes): sigma = 1, inner radius R_L,
    outer R_L + C; every (eta0, R_L) combination in that order."""
    out = []
    for eta0 in etas:
        for rl in radii:
            out.append(dict(geometry=geometry, R_in=rl, R_out=rl + confinement, sigma=1.0,
                            n_cells=int(round(confinement * cells_per_sigma)), beta=0.0, Q_R=Q[0], Q_2=Q[1], Q_3=Q[2],
                            eta0=eta0, T_wall=(1.0, 1.0 + dT), u_wall=(0.0, 0.0), dt=None, precision=precision,
                            chi_model=0))
    return out


def perturbation(shape, seed, amplitude=0.05):
    """Seeded multiplicative perturbation 1 + amplitude * U[-1, 1] of the given shape."""
    rng = np.random.default_rng(seed)
    return 1.0 + amplitude * rng.uniform(-1.0, 1.0, size=shape)
