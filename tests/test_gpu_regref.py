"""The steady regular reflection of a 30-degree Mach-10 shock (Sec. 4.2,
Fig. 11, Eq. Riemann-3) on the GPU: the three states and both shock lines
against the exact oblique-shock solution, and a reduced grid against the
oracle."""
import math

import numpy as np
import pytest

import oracle
from oracle import gasdynamics as gd
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 1.4


def _exact():
    p = W.regular_reflection()
    top = p.sides[3].state_lo
    r, u, v, T = top
    ref = gd.oblique_shock_for_turn(r, u, v, r * T, -math.atan2(v, u), G)
    x_reflect = 3.0 / math.tan(math.pi / 6)                 # incident shock meets the wall
    slope_reflected = math.tan(math.atan2(v, u) + ref[4])    # reflected shock line
    return p, (1.0, r, ref[0]), x_reflect, slope_reflected


def _index(coord, dx):
    return int(round(coord / dx - 0.5))


@pytest.mark.parametrize("prec", ["fp64", "fp32_tdf"])
def test_regular_reflection_matches_exact_solution(prec):
    p, rho, x_ref, slope = _exact()
    with lbm.Lattice(p, prec) as lat:
        lat.init(*W.initial_fields(p)).step(p.steps)
        lat.sync()
        r = lat.moments()[0].double().cpu().numpy()
    dx = p.dx
    # region 1 (inflow), 2 (behind the incident shock), 3 (behind the reflected one)
    assert r[_index(0.5, dx), _index(2.0, dx)] == pytest.approx(rho[0], rel=0.01)
    assert r[_index(2.5, dx), _index(3.0, dx)] == pytest.approx(rho[1], rel=0.02)
    assert r[_index(0.3, dx), _index(8.0, dx)] == pytest.approx(rho[2], rel=0.03)
    # incident shock along y = 1.5: exact x = 1.5 / tan 30
    row = r[_index(1.5, dx)]
    x_inc = (np.argmax(row > 0.5 * (rho[0] + rho[1])) + 0.5) * dx
    assert abs(x_inc - 1.5 / math.tan(math.pi / 6)) <= 3 * dx
    # reflected shock along x = 8: exact y = (8 - x_reflect) tan(angle)
    col = r[:, _index(8.0, dx)]
    y_ref = (np.argmax(col < 0.5 * (rho[1] + rho[2])) + 0.5) * dx
    assert abs(y_ref - (8.0 - x_ref) * slope) <= 4 * dx


def test_regular_reflection_reduced_grid_matches_oracle_fp64():
    p = W.regular_reflection(ny=60, steps=1500)
    oracle.set_threads(oracle.max_threads())
    f = oracle.init(p, *W.initial_fields(p))
    assert oracle.run(p, f, p.steps) == 0
    ref = oracle.fields(p, f)
    with lbm.Lattice(p, "fp64") as lat:
        lat.init(*W.initial_fields(p)).step(p.steps)
        g = [t.cpu().numpy() for t in lat.moments()]
    assert np.max(np.abs(g[0] - ref[0]) / ref[0]) <= 1e-10
    assert np.max(np.abs(g[3] - ref[3]) / ref[3]) <= 1e-10
    U = np.max(np.hypot(ref[1], ref[2]))
    assert max(np.max(np.abs(g[1] - ref[1])), np.max(np.abs(g[2] - ref[2]))) <= 1e-10 * U
