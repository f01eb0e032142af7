"""Brute force on tiny grids: one step of Eq. (SEC-VON-11) written out node
by node in plain Python from the paper's formulas -- moments (Eqs. e4, e5,
e7), equilibrium (Eqs. e16-e18 via the numpy restatement in
oracle/vonneumann.py, independent of the C oracle), the beta-upwind first
derivative of Eqs. (SEC-VON-2a/2b), the central second derivative, and the
BGK relaxation with factor dt / tau -- against the C oracle's step, at every
node and population of a 3 x 3 periodic grid and a 4 x 5 grid with
zero-gradient sides."""
import numpy as np
import pytest

import oracle
from oracle import vonneumann as vn
from paper_0706_0405_gb300 import workloads as W
from paper_0706_0405_gb300.workloads import Side


def _one_step(p, f):
    """f: (9, ny, nx) interior values; returns the next level (9, ny, nx)."""
    vx, vy = vn.velocities(p.c1, p.c2)
    eta2 = np.array([p.eta0 ** 2] + [0.0] * 8)
    periodic = p.sides[0].kind_lo == "periodic"
    ny, nx = f.shape[1:]

    def at(i, y, x):  # the ghost rule: wrap or copy the adjacent node
        if periodic:
            return f[i, y % ny, x % nx]
        return f[i, min(max(y, 0), ny - 1), min(max(x, 0), nx - 1)]

    def deriv(i, y, x, dy, dx, v):  # Eqs. (SEC-VON-2a / 2b) along one axis
        plus, here, minus = at(i, y + dy, x + dx), at(i, y, x), at(i, y - dy, x - dx)
        b = p.beta
        if v >= 0:
            return (b * plus + (1 - 2 * b) * here - (1 - b) * minus) / p.dx
        return ((1 - b) * plus - (1 - 2 * b) * here - b * minus) / p.dx

    out = np.empty_like(f)
    for y in range(ny):
        for x in range(nx):
            fn = f[:, y, x]
            rho = fn.sum()
            ux, uy = (fn * vx).sum() / rho, (fn * vy).sum() / rho
            E = (fn * (vx ** 2 + vy ** 2 + eta2)).sum()
            T = (E / rho - ux ** 2 - uy ** 2) / p.b
            feq = vn.feq_state(rho, ux, uy, T, p.b, p.c1, p.c2, p.eta0)
            for i in range(9):
                adv = vx[i] * deriv(i, y, x, 0, 1, vx[i]) + vy[i] * deriv(i, y, x, 1, 0, vy[i])
                lap = (at(i, y, x + 1) - 2 * fn[i] + at(i, y, x - 1)
                       + at(i, y + 1, x) - 2 * fn[i] + at(i, y - 1, x)) / p.dx ** 2
                out[i, y, x] = (fn[i] - p.dt * adv + p.dt * p.lam[i] * lap
                                + p.dt / p.tau * (feq[i] - fn[i]))
    return out


@pytest.mark.parametrize("nx,ny,kind", [(3, 3, "periodic"), (4, 5, "outflow")])
def test_tiny_grid_step_matches_brute_force(nx, ny, kind):
    rng = np.random.Generator(np.random.PCG64(nx * 10 + ny))
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), c1=3.0, c2=8.0, eta0=5.0, dx=0.05, alpha=0.3,
                  beta=0.3, lam_scale=1.7, sides=(Side(kind),) * 4)
    p = p.with_(tau=p.dt / 0.7)
    base = vn.feq_state(1.1, 0.4, -0.3, 0.9, p.b, p.c1, p.c2, p.eta0)
    f0 = base[:, None, None] * (1.0 + 0.05 * rng.standard_normal((9, ny, nx)))
    state = oracle.empty_state(p)
    oracle.interior(state)[:] = f0
    assert oracle.run(p, state, 1) == 0
    got = oracle.interior(state)
    want = _one_step(p, f0)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
