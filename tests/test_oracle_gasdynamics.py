"""Pins of the oracle's gas-dynamics references (exact Riemann solution and
Rankine-Hugoniot jumps), and of the oracle's runs against them (Sec. 4)."""
import math

import numpy as np
import pytest

import oracle
from oracle import gasdynamics as gd
from paper_0706_0405_gb300 import workloads as W

G = 1.4


def test_regular_reflection_top_state_is_rankine_hugoniot(paper_values):
    """Eq. (Riemann-3): the prescribed top state is the Mach-10 inflow behind a
    30-degree oblique shock, to every digit the paper prints."""
    r, u1, u2, p = paper_values["riemann3_inflow_rho_u1_u2_p"]
    ang = math.radians(paper_values["regular_reflection_angle_deg"][0])
    got = gd.oblique_shock(r, u1, u2, p, (math.sin(ang), math.cos(ang)), G)
    want = paper_values["riemann3_top_rho_u1_u2_p"]
    digits = paper_values["riemann3_top_printed_decimals"]
    for g, w, d in zip(got, want, digits):
        assert round(g, int(d)) == pytest.approx(w, abs=1e-12)
    assert abs(got[2] - want[2]) < 0.5e-4


def test_dmr_post_shock_state():
    """A Mach-10 shock into (rho, p) = (1.4, 1) at rest leaves rho = 8,
    u = 8.25, p = 116.5 exactly (ratio (gamma+1)M^2/((gamma-1)M^2+2) = 40/7)."""
    rho, u, p, s = gd.moving_shock(1.4, 1.0, 10.0, G)
    assert (rho, u, p, s) == pytest.approx((8.0, 8.25, 116.5, 10.0), rel=1e-14)
    post = W.DMR_POST
    assert post[0] == 8.0 and post[3] == 116.5
    assert math.hypot(post[1], post[2]) == pytest.approx(u, rel=1e-15)


def _shock_frame_fluxes(rho1, u1, p1, rho2, u2, p2, s):
    m1, m2 = rho1 * (u1 - s), rho2 * (u2 - s)
    return (m1 - m2, m1 * (u1 - s) + p1 - m2 * (u2 - s) - p2,
            m1 * (G / (G - 1) * p1 / rho1 + 0.5 * (u1 - s) ** 2)
            - m2 * (G / (G - 1) * p2 / rho2 + 0.5 * (u2 - s) ** 2))


@pytest.mark.parametrize("WL,WR", [
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),          # Sod
    ((1000.0, 0.0, 1000.0), (1.0, 0.0, 1.0)),      # Eq. (Riemann-2)
    ((1.4, 30.0, 1.0), (1.4, 0.0, 1.0)),           # Eq. (Riemann-1)
    ((1.4, 3.0, 1.0), (1.4, 0.0, 1.0)),            # Mach-3 tube
    ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),           # two rarefactions
])
def test_riemann_solution_obeys_jump_conditions(WL, WR):
    """Across each shock the mass, momentum and energy fluxes in the shock
    frame are continuous; across each rarefaction u + 2a/(gamma-1) (left) or
    u - 2a/(gamma-1) (right) and p / rho^gamma are constant; p and u are
    continuous at the contact."""
    ps, us = gd.riemann_star(WL, WR, G)
    sl, sr = gd.wave_speeds(WL, WR, G)
    eps = 1e-9
    for (r, u, p), side, s in ((WL, -1, sl), (WR, 1, sr)):
        inner = gd.riemann_sample(WL, WR, G, us + side * eps * (1 + abs(us)))[:, 0]
        if ps > p:  # shock
            fl = _shock_frame_fluxes(r, u, p, *inner, s)
            scale = r * (abs(u) + abs(s) + 1) ** 3 + p * (abs(u) + abs(s) + 1)
            assert max(abs(v) for v in fl) < 1e-9 * scale
        else:
            a = gd.sound_speed(r, p, G)
            ai = gd.sound_speed(inner[0], inner[2], G)
            assert u - side * 2 * a / (G - 1) == pytest.approx(
                inner[1] - side * 2 * ai / (G - 1), rel=1e-10, abs=1e-10)
            assert p / r ** G == pytest.approx(inner[2] / inner[0] ** G, rel=1e-10)
    left = gd.riemann_sample(WL, WR, G, us - 1e-9)[:, 0]
    right = gd.riemann_sample(WL, WR, G, us + 1e-9)[:, 0]
    assert left[2] == pytest.approx(right[2], rel=1e-12) and left[1] == pytest.approx(right[1], rel=1e-9, abs=1e-9)


def test_riemann_symmetric_and_trivial_cases():
    ps, us = gd.riemann_star((1.0, 1.5, 1.0), (1.0, -1.5, 1.0), G)
    assert abs(us) < 1e-13 and ps > 1.0
    ps, us = gd.riemann_star((0.7, 0.3, 2.0), (0.7, 0.3, 2.0), G)
    assert ps == pytest.approx(2.0, rel=1e-13) and us == pytest.approx(0.3, rel=1e-12)


def test_sod_star_state():
    """Widely tabulated exact star state of Sod's tube: p* = 0.30313,
    u* = 0.92745."""
    ps, us = gd.riemann_star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G)
    assert round(ps, 5) == 0.30313 and round(us, 5) == 0.92745


def _tube_error(nx, t_end=0.1, alpha=0.036):
    WL, WR = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    p = W.riemann("sod", nx, 2, 1.0, (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 0.5, 3.0, 9.0,
                  5.0, alpha=alpha, t_end=t_end)
    f = oracle.init(p, *W.initial_fields(p))
    assert oracle.run(p, f, p.steps) == 0
    r, ux, uy, T = oracle.fields(p, f)
    x = (np.arange(nx) + 0.5) * p.dx
    ex = gd.riemann_profile(WL, WR, G, x, 0.5, p.steps * p.dt)
    assert np.max(np.abs(uy)) < 1e-12
    return np.mean(np.abs(r[0] - ex[0])), np.mean(np.abs(r[0] * T[0] - ex[2])), r, ex


@pytest.mark.slow
def test_oracle_sod_converges_to_exact_solution():
    """Refining dx at fixed alpha lowers the L1 error against the exact
    Riemann solution (the scheme's dissipation scales with c1 dx)."""
    oracle.set_threads(oracle.max_threads())
    e = [_tube_error(nx)[:2] for nx in (100, 200, 400)]
    assert e[0][0] > e[1][0] > e[2][0] and e[0][1] > e[1][1] > e[2][1]
    assert e[2][0] < 0.02
    oracle.set_threads(1)


@pytest.mark.slow
def test_oracle_ratio1000_tube_tracks_exact_solution():
    """Eq. (Riemann-2) on the 2000 x 4 grid for a third of its run: positive
    everywhere, and the density follows the exact solution in L1."""
    oracle.set_threads(oracle.max_threads())
    p = W.ratio1000_2000x4()
    p = p.with_(ny=2, steps=p.steps // 3)
    f = oracle.init(p, *W.initial_fields(p))
    assert oracle.run(p, f, p.steps) == 0
    r, ux, uy, T = oracle.fields(p, f)
    x = (np.arange(p.nx) + 0.5) * p.dx
    ex = gd.riemann_profile((1000.0, 0.0, 1000.0), (1.0, 0.0, 1.0), G, x, 2.5, p.steps * p.dt)
    rel_l1 = np.mean(np.abs(r[0] - ex[0])) / np.mean(np.abs(ex[0]))
    assert rel_l1 < 0.03
    oracle.set_threads(1)


@pytest.mark.slow
def test_oracle_steady_mach3_shock_stays_put():
    """A normal Mach-3 shock at rest (upstream Dirichlet, downstream
    zero-gradient, initialised with the Rankine-Hugoniot jump) stays within
    one cell and keeps the downstream state within 1 %."""
    rho1, u1, p1 = 1.4, 3.0, 1.0
    rho2, u2, p2 = gd.normal_shock(rho1, u1, p1, G)
    nx = 200
    p = W.riemann("steady", nx, 2, 1.0, (rho1, u1, 0.0, p1), (rho2, u2, 0.0, p2), 0.5, 4.0, 10.0,
                  6.0, alpha=0.05, steps=2000)
    left = (rho1, u1, 0.0, p1 / rho1)
    p = p.with_(sides=(W.Side("dirichlet", state_lo=left, state_hi=left),) + p.sides[1:])
    f = oracle.init(p, *W.initial_fields(p))
    assert oracle.run(p, f, p.steps) == 0
    r = oracle.fields(p, f)[0][0]
    mid = 0.5 * (rho1 + rho2)
    pos = np.argmax(r > mid)
    assert abs(pos - nx // 2) <= 1
    down = oracle.fields(p, f)
    assert down[0][0, -20] == pytest.approx(rho2, rel=0.01)
    assert down[1][0, -20] == pytest.approx(u2, rel=0.01)
    assert down[0][0, -20] * down[3][0, -20] == pytest.approx(p2, rel=0.01)


def test_oblique_shock_for_turn_inverts_the_incident_shock(paper_values):
    """Turning the Mach-10 inflow by the deflection of the Eq. (Riemann-3) top
    state gives back the 30-degree shock; the reflected shock that turns that
    state back along the wall has the textbook weak-solution angle and leaves
    the flow parallel to the wall."""
    r, u1, u2, p = paper_values["riemann3_inflow_rho_u1_u2_p"]
    top = gd.oblique_shock(r, u1, u2, p, (0.5, math.sqrt(3) / 2), G)
    turn = math.atan2(top[2], top[1])
    inc = gd.oblique_shock_for_turn(r, u1, u2, p, turn, G)
    assert math.degrees(inc[4]) == pytest.approx(paper_values["regular_reflection_angle_deg"][0], abs=1e-9)
    assert inc[:4] == pytest.approx(top, rel=1e-10)
    ref = gd.oblique_shock_for_turn(*top, -turn, G)
    assert abs(ref[2]) < 1e-12 * abs(ref[1])
    # mass flux through the reflected shock is continuous; the shock line
    # leans by beta from the oncoming flow towards the side the flow turns to
    line = math.atan2(top[2], top[1]) + ref[4]
    n = (math.sin(line), -math.cos(line))
    m_in = top[0] * (top[1] * n[0] + top[2] * n[1])
    m_out = ref[0] * (ref[1] * n[0] + ref[2] * n[1])
    assert abs(m_in - m_out) < 1e-9 * abs(m_in)


def test_regular_reflection_states_are_vetted():
    from oracle import vonneumann as vn
    p = W.regular_reflection()
    top = p.sides[3].state_lo
    r, u, v, T = top
    ref = gd.oblique_shock_for_turn(r, u, v, r * T, -math.atan2(v, u), G)
    states = [p.setup["state"], top, (ref[0], ref[1], ref[2], ref[3] / ref[0])]
    for st in states:
        g = vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta, np.array(p.lam))
        assert g <= 1.0 + 1e-9, (st, g)
