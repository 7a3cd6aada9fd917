"""Pins of the oracle's dense-gas closure (Sec. II) against the paper's Table I and
textbook identities."""
import math
import os

import numpy as np
import pytest

from oracle import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_kn.txt")


def _table1():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            C, eta0, kn = line.split()
            rows.append((float(C), float(eta0), kn))
    return rows


def test_table1_knudsen_numbers_reproduced_to_printed_digits():
    rows = _table1()
    assert len(rows) == 9
    for C, eta0, kn in rows:
        digits = len(kn.split(".")[1])
        assert round(model.knudsen(C, eta0), digits) == pytest.approx(float(kn), abs=0.5 * 10 ** -digits)
        # and the inverse relation used to set sigma from Kn
        assert model.confinement(model.knudsen(C, eta0), eta0) == pytest.approx(C, rel=1e-14)


def test_chi_matches_carnahan_starling_equation_of_state():
    # chi = (P/(n T) - 1)/(n b), n b = 4 eta, with the Carnahan-Starling compressibility
    # Z = (1 + eta + eta^2 - eta^3)/(1 - eta)^3 (Eq. chi, first equality).
    eta = np.linspace(1e-4, 0.45, 50)
    Z = (1 + eta + eta ** 2 - eta ** 3) / (1 - eta) ** 3
    assert np.allclose(model.chi_set(eta), (Z - 1) / (4 * eta), rtol=1e-12)
    assert float(model.chi_set(0.0)) == 1.0  # sigma -> 0 recovers Boltzmann (chi -> 1)


def test_prandtl_dilute_limit_and_consistency_with_mu_lambda():
    sigma = 0.3
    n = np.array([1e-9, 1.0, 10.0, 30.0])
    T = np.array([1.0, 1.3, 0.9, 1.1])
    chi = model.chi_set(model.eta_of_n(n, sigma))
    Pr = model.prandtl(n, chi, sigma)
    assert Pr[0] == pytest.approx(2.0 / 3.0, rel=1e-8)
    # lambda = (5/2) mu / Pr  (Eq. viscosity, second line: lambda = c_P tau P_i / Pr)
    mu = model.viscosity(n, T, chi, sigma)
    lam = model.conductivity(n, T, chi, sigma)
    assert np.allclose(Pr, 2.5 * mu / lam, rtol=1e-13)


def test_hard_sphere_dilute_transport_coefficients():
    # chi -> 1 and b rho -> 0: mu -> mu0 = 5/(16 sigma^2) sqrt(T/pi) (Eq. viscosity)
    sigma, T = 0.7, 1.7
    mu = model.viscosity(1e-12, T, 1.0, sigma)
    assert mu == pytest.approx(5.0 / (16.0 * sigma ** 2) * math.sqrt(T / math.pi), rel=1e-10)


def test_physical_parameters_from_kn():
    C, sigma, n0 = model.physical_parameters(0.1, 0.1, 1.0)
    assert sigma == pytest.approx(1.0 / C)
    assert model.eta_of_n(n0, sigma) == pytest.approx(0.1, rel=1e-14)
