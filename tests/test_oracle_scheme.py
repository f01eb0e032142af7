"""Pins of the oracle's time step (Eqs. SEC-VON-1, 2a-2d, 11) and boundary
layer: invariances, conservation, closed-form Fourier response, the
linearised step against the amplification matrix (Eqs. SEC-VON-8, 9, 12),
relaxation, and the mirror symmetry of the reflecting wall."""
import math

import numpy as np
import pytest

import oracle
from oracle import vonneumann as vn
from paper_0706_0405_gb300 import workloads as W
from paper_0706_0405_gb300.workloads import Side


def _run_copy(p, f, n, n0=0):
    g = f.copy()
    bad = oracle.run(p, g, n, n0)
    return g, bad


@pytest.mark.parametrize("sides,state", [
    ((Side("periodic"),) * 4, (1.3, 2.1, -1.7, 0.8)),          # Galilean-shifted
    ((Side("outflow"),) * 4, (0.7, -1.1, 0.6, 1.9)),
    ((Side("dirichlet", state_lo=(2.0, 0.9, 0.3, 1.1)),) * 4, (2.0, 0.9, 0.3, 1.1)),
    ((Side("outflow"), Side("outflow"), Side("reflect"), Side("reflect")), (1.0, 1.5, 0.0, 1.0)),
    ((Side("reflect"), Side("reflect"), Side("periodic"), Side("periodic")), (1.0, 0.0, 0.8, 1.0)),
])
def test_uniform_state_is_fixed(sides, state):
    p = W.uniform(13, 7, state, sides=sides)
    f = oracle.init(p, *W.initial_fields(p))
    g, bad = _run_copy(p, f, 1000)
    assert bad == 0
    fi, gi = oracle.interior(f), oracle.interior(g)
    assert np.max(np.abs(gi - fi)) <= 1e-12 * np.max(np.abs(fi))


def _smooth_periodic(nx, ny, c1=3.0, c2=9.0, eta0=5.0, alpha=0.05, seed=0):
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), c1=c1, c2=c2, eta0=eta0, alpha=alpha)
    x, y = W.centres(p)
    L, H = nx * p.dx, ny * p.dx
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(-1, 1, 8)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x / L + a[0]) * np.cos(2 * np.pi * y / H + a[1])
    ux = 0.5 + 0.3 * np.cos(2 * np.pi * x / L + a[2])
    uy = -0.2 + 0.3 * np.sin(4 * np.pi * y / H + a[3])
    T = 1.0 + 0.2 * np.cos(2 * np.pi * (x / L + y / H) + a[4])
    return p, (rho, ux, uy, T)


def test_periodic_conservation():
    """The beta-upwind weights (beta, 1 - 2 beta, -(1 - beta)) and the
    Laplacian weights (1, -2, 1) each sum to zero, so on a periodic grid the
    stencil only moves mass, momentum and energy between nodes; the collision
    keeps them by Eqs. (e4), (e5), (e7)."""
    p, flds = _smooth_periodic(24, 16)
    f = oracle.init(p, *flds)
    s0 = oracle.sums(p, f)
    g, bad = _run_copy(p, f, 600)
    assert bad == 0
    s1 = oracle.sums(p, g)
    scale = np.array([s0[0], s0[0] * 9.0, s0[0] * 9.0, s0[3]])
    assert np.all(np.abs(s1 - s0) <= 1e-12 * scale), (s1 - s0) / scale
    # and the state did change
    assert np.max(np.abs(oracle.interior(g) - oracle.interior(f))) > 1e-3


@pytest.mark.parametrize("beta", [0.0, 0.25, 0.5])
def test_pure_advection_matches_closed_form(beta):
    """With the collision off (dt / tau = 0) and no dissipation each
    population is advected alone, and a Fourier mode exp(i k x) is multiplied
    per step by 1 - (v dt / dx) phi(k dx), phi of Eq. (SEC-VON-9); beta = 0 is
    the first-order upwind scheme and beta = 1/2 the central one (Sec. 2)."""
    nx, ny, m = 32, 16, 3
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), alpha=0.3, beta=beta)
    p = p.with_(tau=1e300, lam=(0.0,) * 9)
    x, y = W.centres(p)
    kx, ky = 2 * np.pi * m / (nx * p.dx), 2 * np.pi * 2 / (ny * p.dx)
    f = oracle.empty_state(p)
    eps = 1e-3
    for i in range(9):
        oracle.interior(f)[i] = 1.0 + eps * np.cos(kx * x + ky * y + 0.3 * i)
    g, _ = _run_copy(p, f, 1)
    vx, vy = oracle.velocities(p.c1, p.c2)
    for i in range(9):
        gain = 1.0 - (p.dt / p.dx) * (vx[i] * vn.phi(kx * p.dx, vn.SX[i], beta)
                                      + vy[i] * vn.phi(ky * p.dx, vn.SY[i], beta))
        want = 1.0 + eps * np.real(gain * np.exp(1j * (kx * x + ky * y + 0.3 * i)))
        assert np.max(np.abs(oracle.interior(g)[i] - want)) <= 1e-14, i
    if beta == 0.0:
        d = (1.0 - np.cos(kx * p.dx)) + 1j * np.sin(kx * p.dx)   # (f0 - f_-) for v > 0
        assert abs(vn.phi(kx * p.dx, 1, 0.0) - d) < 1e-15
    if beta == 0.5:
        assert abs(vn.phi(kx * p.dx, 1, 0.5) - 1j * np.sin(kx * p.dx)) < 1e-15


def test_upwind_is_monotone():
    """beta = 0 with |v| dt / dx <= 1 never creates a new extremum; upwinding
    against the flow would."""
    nx = 64
    p = W.uniform(nx, 2, (1.0, 0.0, 0.0, 1.0), alpha=0.9, beta=0.0)
    p = p.with_(tau=1e300, lam=(0.0,) * 9)
    f = oracle.empty_state(p)
    for i in range(9):
        oracle.interior(f)[i] = np.where((np.arange(nx) > 20) & (np.arange(nx) < 40), 2.0, 1.0)
    g, _ = _run_copy(p, f, 40)
    assert oracle.interior(g).max() <= 2.0 + 1e-13 and oracle.interior(g).min() >= 1.0 - 1e-13


def test_dissipation_closed_form():
    """Population 0 (v = 0) with the collision off sees only the dissipation
    term: a mode decays by 1 - lambda_0 dt / dx^2 (4 - 2 cos kx dx - 2 cos ky dx)
    per step (last term of Eq. SEC-VON-12)."""
    nx, ny = 20, 12
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), alpha=0.3, lam_scale=3.0)
    p = p.with_(tau=1e300)
    x, y = W.centres(p)
    kx, ky = 2 * np.pi * 2 / (nx * p.dx), 2 * np.pi / (ny * p.dx)
    f = oracle.empty_state(p)
    oracle.interior(f)[:] = 1.0
    oracle.interior(f)[0] = 1.0 + 1e-2 * np.cos(kx * x + ky * y)
    g, _ = _run_copy(p, f, 1)
    decay = 1.0 - p.lam[0] * p.dt / p.dx ** 2 * (4.0 - 2 * np.cos(kx * p.dx) - 2 * np.cos(ky * p.dx))
    want = 1.0 + 1e-2 * decay * np.cos(kx * x + ky * y)
    assert np.max(np.abs(oracle.interior(g)[0] - want)) < 1e-15


@pytest.mark.parametrize("omega", [1.0, 0.37])
def test_relaxation_factor_is_dt_over_tau(omega):
    """A spatially uniform, non-equilibrium f on a periodic grid feels only the
    collision: f -> f + (dt / tau) (f^eq(moments f) - f) (Eq. SEC-VON-1 with
    dt = epsilon), keeping rho, rho u and the energy."""
    p = W.uniform(5, 3, (1.0, 0.0, 0.0, 1.0))
    p = p.with_(tau=p.dt / omega)
    rng = np.random.Generator(np.random.PCG64(5))
    f9 = oracle.feq(p, 1.2, 0.3, -0.4, 0.9) * (1 + 0.05 * rng.standard_normal(9))
    f = oracle.empty_state(p)
    oracle.interior(f)[:] = f9[:, None, None]
    g, _ = _run_copy(p, f, 1)
    m = oracle.moments(p, f9)
    want = f9 + omega * (oracle.feq(p, *m) - f9)
    got = oracle.interior(g)[:, 1, 2]
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(f9))
    assert np.allclose(oracle.moments(p, got), m, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("state,kv", [
    ((1.0, 0.8, -0.3, 1.0), (3, 1)),
    ((1.0, 2.0, 0.0, 0.5), (1, 2)),
    ((2.0, -1.0, 1.5, 2.0), (5, 7)),
])
def test_linearised_step_equals_amplification_matrix(state, kv):
    """One oracle step applied to f^eq(state) + eps F exp(i k.x) (central
    difference in eps) must give G(k) F of Eqs. (SEC-VON-8, 9, 12), column by
    column: the C step and the numpy G are written independently."""
    nx = ny = 16
    p = W.uniform(nx, ny, state, alpha=0.2, lam_scale=1.5)
    p = p.with_(tau=p.dt / 0.8)
    x, y = W.centres(p)
    kx, ky = 2 * np.pi * kv[0] / (nx * p.dx), 2 * np.pi * kv[1] / (ny * p.dx)
    base = oracle.feq(p, *state)
    G = vn.amplification_matrix(kx * p.dx, ky * p.dx, state, p.b, p.c1, p.c2, p.eta0, p.dt,
                                p.dx, p.tau, p.beta, np.array(p.lam))
    ph = np.exp(1j * (kx * x + ky * y))
    eps = 1e-6
    for j in range(9):
        outs = []
        for sgn in (+1, -1):
            f = oracle.empty_state(p)
            oracle.interior(f)[:] = base[:, None, None]
            oracle.interior(f)[j] += sgn * eps * np.real(ph)
            g, _ = _run_copy(p, f, 1)
            outs.append(oracle.interior(g).copy())
        resp = (outs[0] - outs[1]) / (2 * eps)           # (9, ny, nx), real part of G F e^{ikx}
        want = np.real(G[:, j][:, None, None] * ph[None])
        assert np.max(np.abs(resp - want)) < 1e-7 * max(1.0, np.abs(G).max()), j


def test_reflecting_wall_is_a_mirror():
    """A reflecting wall at y = 0 must give the same interior as the
    symmetric continuation: a periodic grid of twice the height holding the
    data and its mirror image (v_y reversed)."""
    nx, ny = 12, 6
    p, flds = _smooth_periodic(nx, 2 * ny, seed=4)
    rho, ux, uy, T = [a[:ny] for a in flds]
    walled = p.with_(ny=ny, sides=(Side("periodic"), Side("periodic"), Side("reflect"),
                                   Side("reflect")))
    f = oracle.init(walled, rho, ux, uy, T)
    g, _ = _run_copy(walled, f, 50)
    full = p.with_(ny=2 * ny)
    mir = lambda a: np.concatenate([a[::-1], a])
    h = oracle.init(full, mir(rho), mir(ux), np.concatenate([-uy[::-1], uy]), mir(T))
    h2, _ = _run_copy(full, h, 50)
    top = oracle.interior(h2)[:, ny:, :]
    assert np.max(np.abs(oracle.interior(g) - top)) < 1e-13 * np.abs(top).max()


def test_periodic_shift_invariance():
    p, flds = _smooth_periodic(20, 10, seed=9)
    f = oracle.init(p, *flds)
    g, _ = _run_copy(p, f, 30)
    h = oracle.init(p, *[np.roll(a, (3, 5), axis=(0, 1)) for a in flds])
    h2, _ = _run_copy(p, h, 30)
    assert np.array_equal(np.roll(oracle.interior(g), (3, 5), axis=(1, 2)), oracle.interior(h2))


def test_ghost_layer_kinds():
    """Ghost rules: outflow copies the adjacent node, Dirichlet holds f^eq of
    its state, a split side switches at split0 + split_speed t (strictly
    below the split uses the 'lo' kind), corners stay unread (NaN)."""
    nx, ny = 8, 5
    post, pre = (8.0, 7.0, -4.0, 14.0), (1.4, 0.0, 0.0, 0.7)
    sides = (Side("outflow"), Side("dirichlet", state_lo=pre, state_hi=pre),
             Side("dirichlet", "reflect", 0.3, 0.0, post, post),
             Side("dirichlet", "dirichlet", 0.2, 2.0, post, pre))
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), dx=0.1, sides=sides)
    rng = np.random.Generator(np.random.PCG64(1))
    f = oracle.empty_state(p)
    oracle.interior(f)[:] = rng.uniform(0.5, 1.5, (9, ny, nx))
    t = 0.1                                    # top split at 0.2 + 0.2 = 0.4
    oracle.fill_ghosts(p, f, t)
    assert np.array_equal(f[:, 1:-1, 0], f[:, 1:-1, 1])                       # outflow
    assert np.allclose(f[:, 1:-1, -1], oracle.feq(p, *pre)[:, None])          # Dirichlet
    xs = (np.arange(nx) + 0.5) * p.dx
    for j, x in enumerate(xs):
        top = f[:, -1, j + 1]
        assert np.allclose(top, oracle.feq(p, *(post if x < 0.4 else pre)))
        bot = f[:, 0, j + 1]
        if x < 0.3:
            assert np.allclose(bot, oracle.feq(p, *post))
        else:                                     # mirror: 2<->4, 5<->8, 6<->7
            assert np.array_equal(bot, f[[0, 1, 4, 3, 2, 8, 7, 6, 5], 1, j + 1])
    assert np.all(np.isnan(f[:, [0, 0, -1, -1], [0, -1, 0, -1]]))


def test_corner_ghosts_never_read():
    p = W.dmr(16, steps=20)
    f = oracle.init(p, *W.initial_fields(p))
    g, bad = _run_copy(p, f, 20)
    assert bad == 0 and np.all(np.isfinite(oracle.interior(g)))


def test_step_nodes_matches_full_step():
    p = W.dmr(16)
    f = oracle.init(p, *W.initial_fields(p))
    oracle.run(p, f, 7)
    g, _ = _run_copy(p, f, 1, 7)
    nodes = np.array([0, 5, p.nx - 1, p.nx * 3 + 17, p.nodes - 1, p.nodes - p.nx])
    out = oracle.step_nodes(p, f.copy(), 7, nodes)
    gi = oracle.interior(g).reshape(9, -1)
    assert np.array_equal(out, gi[:, nodes].T)


def test_paper_dmr_constants_go_nonphysical_but_the_vetted_set_does_not():
    """Sec. 4.2, Fig. 12: on the paper's 400 x 100 grid with the wall from 20
    mesh lengths, its constants (c1 = 8, c2 = 16, eta0 = 10, dt = 2e-4,
    lambda of Eq. 13) leave nodes with rho <= 0 or T <= 0 within 200 steps
    (t = 0.04); the vetted set (c1 = 10, c2 = 20, eta0 = 15, alpha = 0.1,
    lambda = 2 x Eq. 13) runs the same 0.04 in time cleanly."""
    oracle.set_threads(oracle.max_threads())
    bad = W.dmr_paper(c1=8.0, c2=16.0, eta0=10.0, dt=2e-4, lam_scale=1.0, steps=200)
    f = oracle.init(bad, *W.initial_fields(bad))
    assert oracle.run(bad, f, bad.steps) > 0
    good = W.dmr_paper(t_end=0.04)
    f = oracle.init(good, *W.initial_fields(good))
    assert oracle.run(good, f, good.steps) == 0


def test_fp32_storage_run_is_the_fp64_step_rounded_to_fp32():
    """The FP32-storage run (the error floor of any implementation that
    stores f in FP32): from a state that is already FP32-exact, with sides
    whose ghosts are copies of interior values (periodic, outflow), one step
    is exactly the plain FP64 step with every value rounded to FP32."""
    rng = np.random.Generator(np.random.PCG64(11))
    sides = (Side("periodic"), Side("periodic"), Side("outflow"), Side("outflow"))
    p = W.uniform(23, 9, (1.0, 0.0, 0.0, 1.0), dx=0.01, alpha=0.1, sides=sides, steps=1)
    fields = (1.0 + 0.3 * rng.random((9, 23)), 0.4 * rng.standard_normal((9, 23)),
              0.4 * rng.standard_normal((9, 23)), 1.0 + 0.3 * rng.random((9, 23)))
    f = oracle.init(p, *fields)
    oracle.interior(f)[:] = oracle.interior(f).astype(np.float32).astype(np.float64)
    got, want = f.copy(), f.copy()
    assert oracle.run(p, got, 1, 0, f32_storage=True) == 0
    assert oracle.run(p, want, 1, 0) == 0
    gi, wi = oracle.interior(got), oracle.interior(want)
    assert not np.array_equal(wi, wi.astype(np.float32))  # the plain step leaves FP32
    assert np.array_equal(gi, wi.astype(np.float32).astype(np.float64))
