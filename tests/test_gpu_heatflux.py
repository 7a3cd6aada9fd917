"""The heat-flux channel constants of steady Fourier flow (Sec. IV, comparison of the geometries):
the energy balance makes q_R R constant across the gap between cylinders and q_r r^2 constant
between spheres; the constant, scaled by the inner radius (q_R R / R_L, q_r r^2 / R_L^2), moves
monotonically toward the planar-wall value as the inner radius grows (R_L = 1 .. 50), and grows
with the density.  sigma = 1, C = 4, walls at T = 1 and 1.1, 24 cells per sigma, FP64, each
geometry one batch of 18 instances run to steady state."""
import numpy as np
import pytest

from paper_2403_15051_gb300 import build as fbuild
from paper_2403_15051_gb300 import fdlb
from paper_2403_15051_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()


@pytest.mark.parametrize("geom", [wl.CYL, wl.SPH])
def test_heat_flux_channel_constants(geom):
    ds = wl.heatflux_instances(geom)
    S = fdlb.Solver(ds)
    rc, steps, res = S.run_to_steady(tol=1e-8, max_steps=40_000, check_every=500)
    # a few instances settle on a small oscillation just above the tolerance
    assert np.all(res <= 1e-7), res
    power = 1 if geom == wl.CYL else 2
    const = {}
    for q, d in enumerate(ds):
        info = S.info(q)
        Rc, _, _, _ = fdlb.grid(geom, d["R_in"], d["R_out"], info["sigma"], d["n_cells"])
        qR = S.moments(q)["q1"]
        inner = (Rc - info["R_first"] > 1.0) & (info["R_last"] - Rc > 1.0)  # a sigma from each wall
        c = qR[inner] * Rc[inner] ** power
        assert np.all(c < 0), (q, c)  # heat flows inwards, from the hotter outer wall (T = 1.1)
        spread = (c.max() - c.min()) / abs(c.mean())
        assert spread < 1e-3, (d["eta0"], d["R_in"], spread)
        const[(d["eta0"], d["R_in"])] = c.mean() / d["R_in"] ** power
    print("geometry", geom, {k: round(v, 6) for k, v in const.items()})
    for eta0 in (0.01, 0.1, 0.2):
        v = np.array([abs(const[(eta0, rl)]) for rl in (1.0, 2.0, 5.0, 10.0, 20.0, 50.0)])
        assert np.all(np.diff(v) < 0), (eta0, v)  # toward the planar value, monotonically
    for rl in (1.0, 5.0, 50.0):
        assert abs(const[(0.2, rl)]) > abs(const[(0.1, rl)]) > abs(const[(0.01, rl)])
