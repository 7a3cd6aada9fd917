"""Shared helpers of the tests: the same workload dictionary turned into an oracle problem and
into library parameters, seeded inputs and per-moment comparison scales."""
import os

import numpy as np

from oracle import model as omodel
from oracle import solver as osolver
from paper_2403_15051_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def accept_kn(kn, eta0):
    """C >= 3 under Kn = 1/(6 sqrt2 eta0 chi(eta0) C) (oracle side of the acceptance test)."""
    return omodel.confinement(kn, eta0) >= 3.0


def small_case(geometry=wl.CYL, precision="fp64", n_cells=24, Q=(4, 4, 4), beta=0.0, chi_model=0,
               T_wall=(1.0, 1.2), u_wall=(0.15, 0.0), eta0=0.2, Kn=0.1, R=(1.0, 2.0), dt=None):
    if geometry == wl.SPH:
        u_wall = (0.0, 0.0)
    return dict(geometry=geometry, R_in=R[0], R_out=R[1], n_cells=n_cells, beta=beta, Q_R=Q[0], Q_2=Q[1], Q_3=Q[2],
                Kn=Kn, eta0=eta0, T_wall=T_wall, u_wall=u_wall, dt=dt, precision=precision, chi_model=chi_model)


def oracle_problem(d):
    reduced = d["geometry"] == wl.CYL_Z
    return osolver.make_problem(wl.CYL if reduced else d["geometry"], d["R_in"], d["R_out"], d["n_cells"], d["Q_R"],
                                d["Q_2"], d["Q_3"], reduced=reduced,
                                eta0=d["eta0"], Kn=d.get("Kn"), sigma=d.get("sigma"), beta=d.get("beta", 0.0) or 0.0,
                                chi_model=d.get("chi_model", 0), T_wall=tuple(d["T_wall"]),
                                u_wall=tuple(d["u_wall"]), dt=d.get("dt"), cfl=d.get("cfl") or 0.4)


def perturbed_state(P, seed=11, amp=0.05):
    """Uniform equilibrium of the oracle problem times a seeded perturbation."""
    return osolver.uniform_state(P) * wl.perturbation(P.shape, seed, amp)


def moment_scales(P):
    T0 = 0.5 * (P.T_wall[0] + P.T_wall[1])
    return {"n": P.n0, "u": np.sqrt(T0), "T": T0, "q": P.n0 * T0 ** 1.5}


def compare_moments(m_gpu, m_or, P):
    """Largest |difference| of each moment family divided by its scale (n0, sqrt T0, T0, n0 T0^1.5)."""
    sc = moment_scales(P)
    out = {}
    out["n"] = np.max(np.abs(m_gpu["n"] - m_or["n"])) / sc["n"]
    out["u"] = max(np.max(np.abs(m_gpu[f"u{a + 1}"] - m_or["u"][:, a])) for a in range(3)) / sc["u"]
    out["T"] = np.max(np.abs(m_gpu["T"] - m_or["T"])) / sc["T"]
    out["q"] = max(np.max(np.abs(m_gpu[f"q{a + 1}"] - m_or["q"][:, a])) for a in range(3)) / sc["q"]
    return out
