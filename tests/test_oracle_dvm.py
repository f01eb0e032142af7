"""Pins of the oracle's discrete-velocity model (Sec. 2 of the paper): the
velocity table (Eq. e14), the equilibrium (Eqs. e16-e18) and the moments
(Eqs. e4, e5, e7) against the moment constraints the paper imposes
(Eqs. e4-e8), which the equilibrium must satisfy exactly."""
import math

import numpy as np
import pytest

import oracle
from oracle import vonneumann as vn
from paper_0706_0405_gb300 import workloads as W


def _problem(b=5.0, c1=3.0, c2=9.0, eta0=5.0):
    p = W.uniform(4, 4, (1.0, 0.0, 0.0, 1.0), c1=c1, c2=c2, eta0=eta0)
    return p.with_(b=b)


def _random_cases(n=40, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(n):
        c1 = rng.uniform(1.0, 30.0)
        c2 = c1 * rng.uniform(1.2, 3.5)
        eta0 = rng.uniform(1.0, 40.0)
        b = rng.uniform(2.5, 8.0)
        rho = math.exp(rng.uniform(-3, 7))
        T = math.exp(rng.uniform(-2, 3))
        ux, uy = rng.uniform(-1.2, 1.2, 2) * c1
        yield b, c1, c2, eta0, rho, ux, uy, T


def test_velocity_table_is_eq14_with_cos_sin_diagonals():
    c1, c2 = 3.0, 9.0
    vx, vy = oracle.velocities(c1, c2)
    assert vx[0] == 0.0 and vy[0] == 0.0
    for i in range(1, 5):  # c1 (cos(pi (i+1)/2), sin(pi (i+1)/2))
        th = math.pi * (i + 1) / 2
        assert vx[i] == pytest.approx(c1 * math.cos(th), abs=1e-14)
        assert vy[i] == pytest.approx(c1 * math.sin(th), abs=1e-14)
    for i in range(5, 9):  # c2 (cos(pi ((i+1)/2 + 1/4)), sin(...))
        th = math.pi * ((i + 1) / 2 + 0.25)
        assert vx[i] == pytest.approx(c2 * math.cos(th), abs=1e-14)
        assert vy[i] == pytest.approx(c2 * math.sin(th), abs=1e-14)
    pts = {(round(a, 12), round(b, 12)) for a, b in zip(vx, vy)}
    assert len(pts) == 9, "velocities must be distinct"
    # The literal (cos, cos) of Eq. (e14) would repeat a velocity.
    lit = {(round(c2 * math.cos(math.pi * ((i + 1) / 2 + 0.25)), 12),
            round(c2 * math.cos(math.pi * ((i + 1) / 2 + 0.25)), 12)) for i in range(5, 9)}
    assert len(lit) < 4


@pytest.mark.parametrize("case", list(_random_cases()))
def test_feq_satisfies_moment_constraints(case):
    """Eqs. (e4), (e5), (e7), (e6), (e8) hold for f^eq of any state."""
    b, c1, c2, eta0, rho, ux, uy, T = case
    p = _problem(b, c1, c2, eta0)
    f = oracle.feq(p, rho, ux, uy, T)
    vx, vy = oracle.velocities(c1, c2)
    eta2 = np.array([eta0 ** 2] + [0.0] * 8)
    v2 = vx * vx + vy * vy + eta2
    u2 = ux * ux + uy * uy
    P = rho * T
    scale_m = rho * (1.0 + c2 ** 2 + eta0 ** 2) * (1.0 + c2 ** 3)
    checks = [
        (f.sum(), rho, rho),                                               # (e4)
        ((f * vx).sum(), rho * ux, rho * c2),                              # (e5)
        ((f * vy).sum(), rho * uy, rho * c2),
        ((f * v2).sum(), rho * (b * T + u2), scale_m),                     # (e7)
        ((f * vx * vx).sum(), P + rho * ux * ux, scale_m),                 # (e6)
        ((f * vx * vy).sum(), rho * ux * uy, scale_m),
        ((f * vy * vy).sum(), P + rho * uy * uy, scale_m),
        ((f * v2 * vx).sum(), rho * ((b + 2) * T + u2) * ux, scale_m),     # (e8)
        ((f * v2 * vy).sum(), rho * ((b + 2) * T + u2) * uy, scale_m),
    ]
    for got, want, scale in checks:
        assert abs(got - want) <= 1e-13 * max(abs(want), scale), (got, want)


def test_printed_A0_breaks_mass_constraint():
    """The printed A_0 = (b - 2) T / eta0 (Eq. e17) would violate Eq. (e4)
    unless eta0 = 1; the oracle's A_0 = (b - 2) T / eta0^2 satisfies it."""
    b, eta0, rho, T = 5.0, 5.0, 1.3, 0.9
    p = _problem(b, 3.0, 9.0, eta0)
    f = oracle.feq(p, rho, 0.4, -0.2, T)
    assert f[0] == pytest.approx(rho * (b - 2) * T / eta0 ** 2, rel=1e-15)
    printed = f.copy()
    printed[0] = rho * (b - 2) * T / eta0
    assert abs(f.sum() - rho) < 1e-13 * rho
    assert abs(printed.sum() - rho) > 1e-3 * rho


@pytest.mark.parametrize("case", list(_random_cases(20, seed=11)))
def test_moments_invert_feq(case):
    b, c1, c2, eta0, rho, ux, uy, T = case
    p = _problem(b, c1, c2, eta0)
    m = oracle.moments(p, oracle.feq(p, rho, ux, uy, T))
    assert m[0] == pytest.approx(rho, rel=1e-12)
    assert m[1] == pytest.approx(ux, rel=1e-11, abs=1e-12 * c1)
    assert m[2] == pytest.approx(uy, rel=1e-11, abs=1e-12 * c1)
    assert m[3] == pytest.approx(T, rel=1e-10)


def test_moments_invert_feq_at_mach30():
    """Eq. (Riemann-1) left state with the Fig. 8 constants (c1 = 25, c2 = 50,
    eta0 = 30): E / rho = u^2 + b T is 900 + 3.6, so T comes from a
    cancellation; FP64 keeps it to 1e-12."""
    p = _problem(5.0, 25.0, 50.0, 30.0)
    rho, u, T = 1.4, 30.0, 1.0 / 1.4
    m = oracle.moments(p, oracle.feq(p, rho, u, 0.0, T))
    assert m[0] == pytest.approx(rho, rel=1e-13)
    assert m[1] == pytest.approx(u, rel=1e-13)
    assert m[3] == pytest.approx(T, rel=1e-11)


def test_numpy_feq_agrees_with_c_feq():
    """The von Neumann tool's equilibrium (numpy) and the stepping oracle's (C)
    are two writings of Eqs. (e16)-(e18); both are pinned by the constraints
    above, and they must agree."""
    for b, c1, c2, eta0, rho, ux, uy, T in _random_cases(10, seed=3):
        p = _problem(b, c1, c2, eta0)
        a = oracle.feq(p, rho, ux, uy, T)
        bb = vn.feq_state(rho, ux, uy, T, b, c1, c2, eta0)
        scale = np.abs(a).max()
        assert np.max(np.abs(a - bb)) <= 1e-13 * scale


def test_feq_singular_when_c1_equals_c2():
    """A_i and B_i of Eqs. (e17), (e18) divide by c1^2 - c2^2."""
    p = _problem(5.0, 4.0, 4.0, 5.0)
    with np.errstate(all="ignore"):
        f = oracle.feq(p, 1.0, 0.1, 0.0, 1.0)
    assert not np.all(np.isfinite(f))
