"""Dense-gas closure of the simplified Enskog model (paper Sec. II).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Units: m = k_B = 1.
"""
from __future__ import annotations

import math

import numpy as np


def chi_set(eta):
    """Carnahan-Starling contact value chi_SET(eta) = (2 - eta) / (2 (1 - eta)^3)  (Eq. chi)."""
    eta = np.asarray(eta, dtype=np.float64)
    return (2.0 - eta) / (2.0 * (1.0 - eta) ** 3)


def eta_of_n(n, sigma):
    """Reduced density eta = b rho / 4 = pi sigma^3 n / 6 with b = 2 pi sigma^3 / 3 (below Eq. chi)."""
    return math.pi * sigma ** 3 * np.asarray(n, dtype=np.float64) / 6.0


def b_rho(n, sigma):
    """b rho = (2 pi / 3) sigma^3 n  (= 4 eta), m = 1."""
    return 2.0 * math.pi / 3.0 * sigma ** 3 * np.asarray(n, dtype=np.float64)


def knudsen(C, eta0):
    """Kn = 1 / (6 sqrt(2) eta0 chi(eta0) C)  (Sec. II, Knudsen-number equation)."""
    return 1.0 / (6.0 * math.sqrt(2.0) * eta0 * float(chi_set(eta0)) * C)


def confinement(Kn, eta0):
    """C = L / sigma from the same relation, solved for C."""
    return 1.0 / (6.0 * math.sqrt(2.0) * eta0 * float(chi_set(eta0)) * Kn)


def physical_parameters(Kn, eta0, L):
    """(C, sigma, n0) from (Kn, eta0, L):  C from the Kn relation, sigma = L / C,
    n0 = 6 eta0 / (pi sigma^3)  (Sec. II and Sec. IV, C = L / sigma)."""
    C = confinement(Kn, eta0)
    sigma = L / C
    n0 = 6.0 * eta0 / (math.pi * sigma ** 3)
    return C, sigma, n0


def viscosity(n, T, chi, sigma):
    """mu = mu0 [1/chi + 4/5 b rho + 4/25 (1 + 12/pi) (b rho)^2 chi],
    mu0 = 5/(16 sigma^2) sqrt(T/pi)  (Eq. viscosity)."""
    br = b_rho(n, sigma)
    mu0 = 5.0 / (16.0 * sigma ** 2) * np.sqrt(T / math.pi)
    return mu0 * (1.0 / chi + 0.8 * br + 4.0 / 25.0 * (1.0 + 12.0 / math.pi) * br ** 2 * chi)


def conductivity(n, T, chi, sigma):
    """lambda = lambda0 [1/chi + 6/5 b rho + 9/25 (1 + 32/(9 pi)) (b rho)^2 chi],
    lambda0 = 75/(64 sigma^2) sqrt(T/pi)  (Eq. viscosity, second line)."""
    br = b_rho(n, sigma)
    lam0 = 75.0 / (64.0 * sigma ** 2) * np.sqrt(T / math.pi)
    return lam0 * (1.0 / chi + 1.2 * br + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * math.pi)) * br ** 2 * chi)


def prandtl(n, chi, sigma):
    """Pr = 2/3 [1 + 4/5 x + 4/25 (1 + 12/pi) x^2] / [1 + 6/5 x + 9/25 (1 + 32/(9 pi)) x^2],
    x = b rho chi  (Eq. prandtl)."""
    x = b_rho(n, sigma) * chi
    num = 1.0 + 0.8 * x + 4.0 / 25.0 * (1.0 + 12.0 / math.pi) * x ** 2
    den = 1.0 + 1.2 * x + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * math.pi)) * x ** 2
    return 2.0 / 3.0 * num / den


def relaxation_time(n, T, chi, sigma):
    """tau = mu / P_i with P_i = n T  (Eq. tau)."""
    return viscosity(n, T, chi, sigma) / (n * T)
