"""Dense hard-sphere gas at rest between coaxial cylinders and concentric spheres (the appendix on
the stationary gas): eta0 in {0.01, 0.1, 0.2}, inner radius R_L in {1, 3, 5} sigma, confinement
C in {4, 7, 10}, walls at T_w = 1, each geometry one batch run to steady state.  The checks are
the trends the paper states for these profiles: near-flat for the dilute gas, a non-monotonic
profile near the walls whose strength grows with eta0, weaker layering at the inner (convex) wall
than at the outer one, growing with the inner radius (less curvature), and weaker on the sphere
than on the cylinder at the same inner radius."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


def _profiles(geometry):
    ds = wl.layering_instances(geometry)
    S = fdlb.Solver(ds)
    rc, steps, res = S.run_to_steady(tol=1e-6, max_steps=200000, check_every=500)
    assert rc == 0 and np.all(res <= 1e-6)
    out = {}
    for q, d in enumerate(ds):
        n0 = 6.0 * d["eta0"] / np.pi  # sigma = 1
        out[(d["eta0"], d["R_in"], d["R_out"] - d["R_in"])] = S.moments(q)["n"] / n0
    return out


@pytest.fixture(scope="module")
def profiles():
    return {g: _profiles(g) for g in (wl.CYL, wl.SPH)}


@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_layering_trends(profiles, geom):
    P = profiles[geom]
    for (eta0, rl, c), r in P.items():
        assert np.isclose(np.mean(r), 1.0, atol=0.05)  # the mass is the mean density's
        if eta0 == 0.01:
            assert np.max(np.abs(r - 1.0)) < 2e-3  # dilute: flat
    for rl in (1.0, 3.0, 5.0):
        for c in (4.0, 7.0, 10.0):
            dev = [np.max(np.abs(P[(e, rl, c)] - 1.0)) for e in (0.01, 0.1, 0.2)]
            assert dev[0] < dev[1] < dev[2]  # stronger with density
            r = P[(0.2, rl, c)]
            assert r[0] > 1.02 and r[-1] > 1.02 and r.min() < 0.995  # non-monotonic near the walls
            assert r[0] < r[-1]  # weaker at the inner (convex) wall
    for c in (4.0, 7.0, 10.0):
        inner = [P[(0.2, rl, c)][0] for rl in (1.0, 3.0, 5.0)]
        assert inner[0] < inner[1] < inner[2]  # layering grows as the curvature falls


def test_sphere_layers_less_than_cylinder(profiles):
    for c in (4.0, 7.0, 10.0):
        assert profiles[wl.SPH][(0.2, 1.0, c)][0] < profiles[wl.CYL][(0.2, 1.0, c)][0]
