"""The synthetic workloads (CPU): the batch of Riemann tubes follows its
stated recipe and is reproducible, and the double Mach reflection carries
the Rankine-Hugoniot post-shock state the paper prints."""
import math

import numpy as np

from oracle import gasdynamics as gd
from paper_0706_0405_gb300 import workloads as W


def test_batch_of_tubes_follows_its_recipe_and_is_reproducible():
    probs = W.batch_riemann()
    again = W.batch_riemann()
    assert len(probs) == 256
    assert [p.nx for p in probs] == [p.nx for p in again]
    assert [p.setup["left"] for p in probs] == [p.setup["left"] for p in again]
    nx = np.array([p.nx for p in probs])
    assert nx.min() >= 256 and nx.max() <= 4096 and all(p.ny == 4 for p in probs)
    # log-uniform lengths: the median sits near the geometric mean of 256 and 4096
    assert 700 <= np.median(nx) <= 1400
    r = np.array([p.setup["left"][0] for p in probs])
    mach = np.array([p.setup["left"][1] / math.sqrt(1.4) for p in probs])
    assert r.min() >= 1.0 and r.max() <= 1000.0 and mach.min() >= 0.0 and mach.max() <= 30.0
    for p in probs:
        L, R = p.setup["left"], p.setup["right"]
        # states as (rho, u, v, T): p = rho on the left and 1 on the right, so T = 1 on both sides
        assert L[3] == 1.0 and L[2] == 0.0 and R == (1.0, 0.0, 0.0, 1.0)
        assert math.isclose(p.dx, 1.0 / p.nx) and p.tau == p.dt
        assert math.isclose(p.c2, 2.4 * p.c1) and math.isclose(p.eta0, 1.2 * p.c1)
        assert math.isclose(p.dt, 0.05 * p.dx / p.c2)
        # c1 covers the inflow and the exact star velocity of the tube
        WL, WR = (L[0], L[1], L[0] * L[3]), (R[0], R[1], R[0] * R[3])
        _, u_star = gd.riemann_star(WL, WR, 1.4)
        assert p.c1 >= max(3.0, 1.1 * L[1] + 2.0) and p.c1 > u_star
    assert W.batch_riemann(seed=1)[0].nx != probs[0].nx or W.batch_riemann(seed=1)[1].nx != probs[1].nx


def test_double_mach_reflection_post_shock_state_is_the_rankine_hugoniot_one():
    """A Mach-10 shock into (rho, p) = (1.4, 1) (sound speed 1): the state
    behind it, in the frame where the gas ahead is at rest, is
    rho = 8, |u| = 8.25, p = 116.5, the values the workload uses."""
    rho, u, v, p = W.DMR_POST
    assert math.isclose(math.hypot(u, v), 8.25) and rho == 8.0 and p == 116.5
    g = 1.4
    M = 10.0
    rho2 = 1.4 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = 1.0 * (1 + 2 * g / (g + 1) * (M * M - 1))
    u2 = 10.0 * (1 - 1.4 / rho2)
    assert math.isclose(rho2, 8.0, rel_tol=1e-12)
    assert math.isclose(p2, 116.5, rel_tol=1e-12)
    assert math.isclose(u2, 8.25, rel_tol=1e-12)
