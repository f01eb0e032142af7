"""Reference solutions of the Euler equations (Eq. e2 of the paper) for an ideal
gas with P = rho T (R = 1) and gamma = (b + 2) / b.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

* ``riemann_star`` / ``riemann_sample``: the exact solution of the
  one-dimensional Riemann problem (used for the paper's Eqs. Riemann-1 and
  Riemann-2 and the Sod tube).  The star pressure is the root of
  f_L(p) + f_R(p) + u_R - u_L = 0 with the shock branch
  f_K = (p - p_K) sqrt(A_K / (p + B_K)), A_K = 2 / ((gamma + 1) rho_K),
  B_K = p_K (gamma - 1) / (gamma + 1), and the rarefaction branch
  f_K = 2 a_K / (gamma - 1) ((p / p_K)^((gamma - 1) / (2 gamma)) - 1).
* ``normal_shock`` / ``oblique_shock`` / ``moving_shock``: Rankine-Hugoniot
  jumps (used for Eq. Riemann-3 and the double-Mach-reflection states).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq


def sound_speed(rho, p, gamma):
    return np.sqrt(gamma * p / rho)


def _f_side(p, rho, pk, gamma):
    a = sound_speed(rho, pk, gamma)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * a / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def riemann_star(WL, WR, gamma):
    """Star pressure and velocity for left/right states W = (rho, u, p)."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    al, ar = sound_speed(rl, pl, gamma), sound_speed(rr, pr, gamma)
    if 2.0 / (gamma - 1.0) * (al + ar) <= ur - ul:
        raise ValueError("the data generate a vacuum")
    F = lambda p: _f_side(p, rl, pl, gamma) + _f_side(p, rr, pr, gamma) + ur - ul
    lo, hi = 1e-14 * min(pl, pr), max(pl, pr)
    while F(hi) < 0.0:
        hi *= 2.0
    ps = brentq(F, lo, hi, xtol=1e-15 * hi, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_f_side(ps, rr, pr, gamma) - _f_side(ps, rl, pl, gamma))
    return ps, us


def _sample_left(xi, rl, ul, pl, ps, us, gamma):
    al = sound_speed(rl, pl, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if ps > pl:  # shock
        s = ul - al * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + (gamma - 1.0) / (2.0 * gamma))
        if xi <= s:
            return rl, ul, pl
        return rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps
    head = ul - al
    ast = al * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
    tail = us - ast
    if xi <= head:
        return rl, ul, pl
    if xi >= tail:
        return rl * (ps / pl) ** (1.0 / gamma), us, ps
    u = 2.0 / (gamma + 1.0) * (al + 0.5 * (gamma - 1.0) * ul + xi)
    a = 2.0 / (gamma + 1.0) * (al + 0.5 * (gamma - 1.0) * (ul - xi))
    return rl * (a / al) ** (2.0 / (gamma - 1.0)), u, pl * (a / al) ** (2.0 * gamma / (gamma - 1.0))


def riemann_sample(WL, WR, gamma, xi, star=None):
    """(rho, u, p) of the self-similar solution at xi = (x - x_d) / t."""
    if star is None:
        star = riemann_star(WL, WR, gamma)
    ps, us = star
    xi = np.atleast_1d(np.asarray(xi, dtype=float))
    out = np.zeros((3, xi.size))
    for q, s in enumerate(xi):
        if s <= us:
            out[:, q] = _sample_left(s, *WL, ps, us, gamma)
        else:  # mirror x -> -x of the left-side formulas
            r, u, p = _sample_left(-s, WR[0], -WR[1], WR[2], ps, -us, gamma)
            out[:, q] = (r, -u, p)
    return out


def riemann_profile(WL, WR, gamma, x, x_d, t):
    """Exact (rho, u, p) at positions x and time t > 0 for a diaphragm at x_d."""
    return riemann_sample(WL, WR, gamma, (np.asarray(x) - x_d) / t)


def wave_speeds(WL, WR, gamma):
    """Outermost left and right wave speeds (shock speed or rarefaction head)."""
    ps, us = riemann_star(WL, WR, gamma)
    out = []
    for (r, u, p), sgn in ((WL, -1.0), (WR, 1.0)):
        a = sound_speed(r, p, gamma)
        if ps > p:
            out.append(u + sgn * a * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / p
                                             + (gamma - 1.0) / (2.0 * gamma)))
        else:
            out.append(u + sgn * a)
    return tuple(out)


def normal_shock(rho1, un1, p1, gamma):
    """Downstream (rho, un, p) of a stationary normal shock with upstream normal
    velocity un1 > sound speed."""
    M2 = un1 * un1 / (gamma * p1 / rho1)
    rho2 = rho1 * (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0))
    return rho2, un1 * rho1 / rho2, p2


def oblique_shock(rho1, ux1, uy1, p1, normal, gamma):
    """Downstream (rho, ux, uy, p) of a stationary shock whose unit normal
    ``normal`` points downstream; the tangential velocity is continuous."""
    n = np.asarray(normal, dtype=float)
    n = n / np.linalg.norm(n)
    w1 = ux1 * n[0] + uy1 * n[1]
    rho2, w2, p2 = normal_shock(rho1, w1, p1, gamma)
    return rho2, ux1 - (w1 - w2) * n[0], uy1 - (w1 - w2) * n[1], p2


def moving_shock(rho1, p1, mach, gamma):
    """Shock of Mach number ``mach`` running into gas at rest: returns the
    post-shock (rho, u, p), u along the direction of travel, and the shock
    speed."""
    s = mach * sound_speed(rho1, p1, gamma)
    rho2, w2, p2 = normal_shock(rho1, s, p1, gamma)
    return rho2, s - w2, p2, s


def oblique_shock_for_turn(rho1, ux1, uy1, p1, turn, gamma, strong=False):
    """Stationary oblique shock that turns the flow (ux1, uy1) by the angle
    `turn` (radians, counter-clockwise positive) and its downstream state.
    The shock angle beta (between the upstream velocity and the shock) solves
    tan(turn) = 2 cot(beta) (M^2 sin^2 beta - 1) / (M^2 (gamma + cos 2 beta) + 2);
    the weak root is taken unless strong=True.  Returns (rho, ux, uy, p,
    beta)."""
    speed = float(np.hypot(ux1, uy1))
    M = speed / sound_speed(rho1, p1, gamma)
    th = abs(turn)
    g = lambda b: 2.0 / np.tan(b) * (M * M * np.sin(b) ** 2 - 1.0) / (
        M * M * (gamma + np.cos(2.0 * b)) + 2.0) - np.tan(th)
    mu = np.arcsin(1.0 / M)
    bs = np.linspace(mu + 1e-9, np.pi / 2 - 1e-9, 20001)
    gv = np.array([g(b) for b in bs])
    k = int(np.argmax(gv))
    if gv[k] < 0:
        raise ValueError("turn angle beyond the maximum for this Mach number (detached shock)")
    beta = brentq(g, bs[k], bs[-1]) if strong else brentq(g, bs[0], bs[k])
    # unit normal pointing downstream: the shock line makes angle beta with
    # the flow, on the side the flow turns towards
    phi = np.arctan2(uy1, ux1)
    sgn = 1.0 if turn >= 0 else -1.0
    line = phi + sgn * beta
    n = np.array([np.sin(line), -np.cos(line)]) * sgn
    if n[0] * ux1 + n[1] * uy1 < 0:
        n = -n
    rho2, ux2, uy2, p2 = oblique_shock(rho1, ux1, uy1, p1, n, gamma)
    return rho2, ux2, uy2, p2, beta
