"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Error measures:
  * rho, T: max over nodes of |gpu - oracle| / |oracle|;
  * ux, uy: max |gpu - oracle| / U with U = max(max |u|, max sqrt(T)) of the
    oracle's fields (velocity errors relative to the flow's speed scale);
  * FP64 bar: 1e-10 for all four after the stated step counts;
  * FP32 modes: L1 relative error of rho and T <= 1e-3 across shocks and
    <= 1e-4 on smooth flow, shock position within one cell.
"""
import numpy as np
import pytest

import oracle
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W
from paper_0706_0405_gb300.workloads import Side

pytestmark = pytest.mark.gpu

FP32_MODES = ("fp32", "fp32_t64", "fp32_tdf", "fp32_cons")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(oracle.max_threads())
    yield
    oracle.set_threads(1)


def gpu_run(p, prec, steps=None, fields=None):
    fields = W.initial_fields(p) if fields is None else fields
    with lbm.Lattice(p, prec) as lat:
        lat.init(*fields).step(p.steps if steps is None else steps)
        out = [t.double().cpu().numpy() for t in lat.moments()]
    return out


def oracle_run(p, steps=None, fields=None):
    fields = W.initial_fields(p) if fields is None else fields
    f = oracle.init(p, *fields)
    bad = oracle.run(p, f, p.steps if steps is None else steps)
    assert bad == 0
    return list(oracle.fields(p, f)), f


def max_rel(g, r):
    rho = np.max(np.abs(g[0] - r[0]) / np.abs(r[0]))
    T = np.max(np.abs(g[3] - r[3]) / np.abs(r[3]))
    U = max(np.max(np.abs(r[1])), np.max(np.abs(r[2])), np.sqrt(np.max(r[3])))
    u = max(np.max(np.abs(g[1] - r[1])), np.max(np.abs(g[2] - r[2]))) / U
    return {"rho": rho, "u": u, "T": T}


def l1_rel(a, b):
    return float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))


_CACHE = {}


def cached_oracle(key, p, steps=None):
    if key not in _CACHE:
        _CACHE[key] = oracle_run(p, steps)[0]
    return _CACHE[key]


# ---------------------------------------------------------------- FP64 bar

def test_sod_400x4_fp64_matches_oracle():
    p = W.sod_400x4()
    ref = cached_oracle("sod", p)
    err = max_rel(gpu_run(p, "fp64"), ref)
    assert max(err.values()) <= 1e-10, err


def test_ratio1000_2000x4_fp64_matches_oracle():
    p = W.ratio1000_2000x4()
    ref = cached_oracle("r1000", p)
    err = max_rel(gpu_run(p, "fp64"), ref)
    assert max(err.values()) <= 1e-10, err


def test_dmr_256x64_fp64_matches_oracle():
    """The double Mach reflection (all four boundary kinds, a split wall and
    the moving top split) at reduced size, to t = 0.2."""
    p = W.dmr(64)
    ref = cached_oracle("dmr64", p)
    err = max_rel(gpu_run(p, "fp64"), ref)
    assert max(err.values()) <= 1e-10, err


RAGGED = [
    (1, 1, (Side("periodic"),) * 4),
    (2, 3, (Side("outflow"),) * 4),
    (5, 7, (Side("reflect"), Side("reflect"), Side("reflect"), Side("reflect"))),
    (37, 5, (Side("dirichlet", state_lo=(1.2, 0.3, 0.1, 0.9), state_hi=(1.2, 0.3, 0.1, 0.9)),
             Side("outflow"), Side("dirichlet", "reflect", 0.11, 0.0, (1.5, 0.2, -0.2, 1.1)),
             Side("dirichlet", "outflow", 0.05, 3.0, (0.9, 0.0, -0.3, 1.3)))),
    (131, 67, (Side("periodic"), Side("periodic"), Side("reflect"),
               Side("dirichlet", "dirichlet", 0.4, -0.5, (1.1, 0.5, 0.0, 1.0), (0.8, -0.2, 0.1, 1.2)))),
]


@pytest.mark.parametrize("nx,ny,sides", RAGGED)
def test_ragged_grids_and_boundary_kinds_fp64(nx, ny, sides):
    rng = np.random.Generator(np.random.PCG64(nx * 1000 + ny))
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), dx=0.01, alpha=0.1, sides=sides, steps=60)
    p = p.with_(tau=p.dt / 0.7)
    fields = (1.0 + 0.3 * rng.random((ny, nx)), 0.5 * rng.standard_normal((ny, nx)),
              0.5 * rng.standard_normal((ny, nx)), 1.0 + 0.3 * rng.random((ny, nx)))
    ref = oracle_run(p, fields=fields)[0]
    err = max_rel(gpu_run(p, "fp64", fields=fields), ref)
    assert max(err.values()) <= 1e-11, err


# --------------------------------------------------------------- FP32 modes

def _shock_index(rho, lo, hi):
    mid = 0.5 * (lo + hi)
    return int(np.argmax(rho > mid))


@pytest.mark.parametrize("prec", FP32_MODES)
def test_ratio1000_fp32_modes(prec):
    p = W.ratio1000_2000x4()
    ref = cached_oracle("r1000", p)
    g = gpu_run(p, prec)
    assert l1_rel(g[0], ref[0]) <= 1e-3 and l1_rel(g[3], ref[3]) <= 1e-3
    # the shock runs into the right state (rho = 1); locate it from the right
    rr, rg = ref[0][0][::-1], g[0][0][::-1]
    assert abs(_shock_index(rg, 1.0, 4.0) - _shock_index(rr, 1.0, 4.0)) <= 1


@pytest.mark.parametrize("prec", FP32_MODES)
def test_sod_fp32_modes_smooth_bar(prec):
    p = W.sod_400x4()
    ref = cached_oracle("sod", p)
    g = gpu_run(p, prec)
    assert l1_rel(g[0], ref[0]) <= 1e-4 and l1_rel(g[3], ref[3]) <= 1e-4


@pytest.mark.parametrize("prec", FP32_MODES)
def test_dmr_256x64_fp32_modes(prec):
    p = W.dmr(64)
    ref = cached_oracle("dmr64", p)
    g = gpu_run(p, prec)
    assert l1_rel(g[0], ref[0]) <= 1e-3 and l1_rel(g[3], ref[3]) <= 1e-3


# ----------------------------------------------------- full-size DMR, sampled

def _sample_nodes(p, rng, n=4000):
    nx, ny = p.nx, p.ny
    edge = [0, nx - 1, (ny - 1) * nx, ny * nx - 1]
    edge += list(range(0, nx, 97)) + [(ny - 1) * nx + j for j in range(0, nx, 89)]
    edge += [k * nx for k in range(0, ny, 53)] + [k * nx + nx - 1 for k in range(0, ny, 61)]
    x_wall = int(W.DMR_X0 * ny)  # nodes near the wall start
    edge += [x_wall - 1, x_wall, x_wall + 1]
    return np.unique(np.concatenate([np.array(edge), rng.integers(0, nx * ny, n)]))


@pytest.mark.parametrize("prec", ("fp64",) + FP32_MODES)
def test_dmr_4096x1024_one_step_sampled(prec):
    """At the full 4096 x 1024 size, in the launch configuration the
    benchmark times: after some steps, the GPU's next level at sampled nodes
    (all edges, corners and the wall start included) equals one oracle step
    from the GPU's own level, node by node."""
    import torch
    p = W.dmr(1024)
    n0 = 40
    with lbm.Lattice(p, prec) as lat:
        lat.init(*W.initial_fields(p)).step(n0)
        f0 = lat.get_f().double().cpu().numpy()
        lat.step(1)
        f1 = lat.get_f().double().cpu().numpy()
        torch.cuda.synchronize()
    state = oracle.empty_state(p)
    oracle.interior(state)[:] = f0
    nodes = _sample_nodes(p, np.random.Generator(np.random.PCG64(3)))
    want = oracle.step_nodes(p, state, n0, nodes)            # (count, 9)
    got = f1.reshape(9, -1)[:, nodes].T
    # scale: the largest |f| in the node's star, all populations
    fi = f0.reshape(9, p.ny, p.nx)
    ky, kx = nodes // p.nx, nodes % p.nx
    sc = np.abs(fi[:, ky, kx]).max(axis=0)
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        yy, xx = np.clip(ky + dy, 0, p.ny - 1), np.clip(kx + dx, 0, p.nx - 1)
        sc = np.maximum(sc, np.abs(fi[:, yy, xx]).max(axis=0))
    rtol = 1e-12 if prec == "fp64" else 2e-6
    err = np.abs(got - want) / sc[:, None]
    assert err.max() <= rtol, (prec, err.max(), nodes[np.argmax(err.max(axis=1))])


# ------------------------------------------------- moments, sums, round trips

def test_moments_and_conservation_fp64():
    p = W.dmr(32)
    ref, f = oracle_run(p, steps=200)
    with lbm.Lattice(p, "fp64") as lat:
        lat.init(*W.initial_fields(p)).step(200)
        g = [t.double().cpu().numpy() for t in lat.moments()]
        sums = lat.conservation()
    assert max(max_rel(g, ref).values()) <= 1e-10
    want = oracle.sums(p, f)
    assert np.allclose(sums, want, rtol=1e-13, atol=1e-13 * abs(want[0]))


@pytest.mark.parametrize("prec", FP32_MODES)
def test_conservation_fp32_is_fp64_sum_of_stored_f(prec):
    p = W.dmr(32)
    with lbm.Lattice(p, prec) as lat:
        lat.init(*W.initial_fields(p)).step(50)
        f = lat.get_f().double().cpu().numpy()
        sums = lat.conservation()
    state = oracle.empty_state(p)
    oracle.interior(state)[:] = f
    want = oracle.sums(p, state)
    assert np.allclose(sums, want, rtol=1e-12, atol=1e-12 * abs(want[0]))


def test_periodic_conservation_on_gpu():
    p = W.uniform(96, 64, (1.0, 0.4, -0.3, 1.0), alpha=0.1, steps=500)
    x, y = W.centres(p)
    fields = (1.0 + 0.2 * np.sin(2 * np.pi * x / (96 * p.dx)), np.full_like(x, 0.4),
              -0.3 + 0.1 * np.cos(2 * np.pi * y / (64 * p.dx)), np.ones_like(x))
    with lbm.Lattice(p, "fp64") as lat:
        lat.init(*fields)
        s0 = lat.conservation()
        lat.step(500)
        s1 = lat.conservation()
    assert np.allclose(s1, s0, rtol=1e-12, atol=1e-12 * s0[0])


def test_set_get_save_load_roundtrip():
    import torch
    p = W.dmr(16)
    with lbm.Lattice(p, "fp32") as lat:
        lat.init(*W.initial_fields(p)).step(17)
        assert lat.step_count == 17
        nb = lbm.lbm_checkpoint_bytes(lat.ctx)
        host = np.zeros(nb, dtype=np.uint8)
        lbm.lbm_save(lat.ctx, host, nb)
        dev = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        lbm.lbm_save(lat.ctx, dev, nb)
        assert np.array_equal(host, dev.cpu().numpy())
        f17 = lat.get_f().cpu().numpy()
        lat.step(5)
        f22 = lat.get_f().cpu().numpy()
        lbm.lbm_load(lat.ctx, host, nb)
        assert lat.step_count == 17
        assert np.array_equal(lat.get_f().cpu().numpy(), f17)
        lat.step(5)
        assert np.array_equal(lat.get_f().cpu().numpy(), f22)
        lat.set_f(f17, 17).step(5)
        assert np.array_equal(lat.get_f().cpu().numpy(), f22)
        bad = host.copy()
        bad[8:12] = 0  # nx field
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_load(lat.ctx, bad, nb)
        assert ei.value.status == lbm.LBM_E_INVAL


def test_host_pointers_match_device_pointers():
    p = W.dmr(16)
    fields = [np.ascontiguousarray(a) for a in W.initial_fields(p)]
    with lbm.Lattice(p, "fp64") as lat:
        lbm.lbm_init(lat.ctx, *fields)  # host numpy inputs
        lat.step(30)
        host_out = [np.empty((p.ny, p.nx)) for _ in range(4)]
        lbm.lbm_moments(lat.ctx, *host_out)
        dev_out = [t.cpu().numpy() for t in lat.moments()]
    for a, b in zip(host_out, dev_out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32_tdf"])
def test_page_locked_host_buffers_match_device_buffers(prec):
    """Page-locked host fields are read, and page-locked host moments written,
    in place by the kernels (no staging copy); pageable host memory goes
    through the staging buffer.  All three give the same bits."""
    import torch
    p = W.dmr(16)
    dt = np.float64 if prec == "fp64" else np.float32
    fields = [np.ascontiguousarray(a, dtype=dt) for a in W.initial_fields(p)]
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in fields]
    outs = {}
    for kind in ("pinned", "pageable", "device"):
        with lbm.Lattice(p, prec) as lat:
            if kind == "pinned":
                lbm.lbm_init(lat.ctx, *pinned)
            elif kind == "pageable":
                lbm.lbm_init(lat.ctx, *fields)
            else:
                lat.init(*fields)
            lat.step(30)
            if kind == "device":
                outs[kind] = [t.cpu().numpy() for t in lat.moments()]
            else:
                host = ([torch.empty((p.ny, p.nx), dtype=pinned[0].dtype).pin_memory() for _ in range(4)]
                        if kind == "pinned" else [np.empty((p.ny, p.nx), dtype=dt) for _ in range(4)])
                lbm.lbm_moments(lat.ctx, *host)
                outs[kind] = [np.asarray(h) for h in host]
    for kind in ("pinned", "pageable"):
        for a, b in zip(outs[kind], outs["device"]):
            assert np.array_equal(a, b), kind


def test_nonphysical_state_is_reported():
    """Parameters far outside the von Neumann bound (no dissipation, beta = 0,
    alpha = 0.9, u >> c1) blow up; the status must say so, without a fault."""
    p = W.uniform(64, 8, (1.0, 8.0, 0.0, 0.3), c1=3.0, c2=9.0, eta0=5.0, alpha=0.9, beta=0.0,
                  lam_scale=0.0, steps=4000)
    rng = np.random.Generator(np.random.PCG64(0))
    fields = list(W.initial_fields(p))
    fields[0] = fields[0] * (1 + 1e-3 * rng.standard_normal(fields[0].shape))
    with lbm.Lattice(p, "fp64") as lat:
        lat.init(*fields).step(4000)
        with pytest.raises(lbm.LbmError) as ei:
            lat.sync()
        assert ei.value.status == lbm.LBM_E_NONPHYSICAL
        lat.init(*W.initial_fields(p.with_(setup={"kind": "uniform", "state": (1.0, 0.0, 0.0, 1.0)})))
        lat.sync()  # cleared by lbm_init


def test_step_before_init_is_a_state_error():
    p = W.sod_400x4()
    with lbm.Lattice(p, "fp64") as lat:
        with pytest.raises(lbm.LbmError) as ei:
            lat.step(1)
        assert ei.value.status == lbm.LBM_E_STATE


# ---------------------------------------------------------- launch shapes

SHAPES = [(0, 0, 0, 0), (3, 0, 0, 0), (3, 0, 0, 5), (3, 0, 0, 1), (3, 0, 0, 13), (2, 4, 0, 0), (2, 2, 0, 0),
          (1, 256, 4, 0), (1, 256, 6, 0), (1, 128, 4, 0), (1, 256, 4, 7), (1, 128, 4, 1)]


@pytest.mark.parametrize("prec", FP32_MODES)
@pytest.mark.parametrize("ny", [64, 37])
def test_every_launch_shape_gives_the_same_bits(prec, ny):
    """The thread-per-node kernel, the TMA tile kernel (full wave, 1, 5 and 13
    CTAs; in the double-float mode the CTAs claim their tiles at run time,
    25 launches in a row, so a claim counter not reset between launches
    would show, and with 1 and 5 CTAs, 8 or more tiles each, they claim
    ahead of the copies),
    the vectorised kernel (2 and 4 nodes per thread) and every shape of the
    strip-marching ring kernel (including a grid of 1 and 7 CTAs), on a grid
    whose width is not a multiple of any tile, vector or strip width, do the
    same explicitly rounded arithmetic in the same order, so their levels
    agree bit for bit, edges included."""
    p = W.dmr(ny).with_(nx=4 * ny + 3) if ny == 37 else W.dmr(ny)
    if ny == 37:
        p = p.with_(sides=(p.sides[0], W.Side("periodic"), p.sides[2], p.sides[3]))
        p = p.with_(sides=(W.Side("periodic"),) + p.sides[1:])
    outs = []
    for shape in SHAPES:
        with lbm.Lattice(p, prec) as lat:
            lbm.lbm_set_launch(lat.ctx, *shape)
            lat.init(*W.initial_fields(p)).step(25)
            outs.append(lat.get_f().cpu().numpy())
            lat.sync()
    for s, o in zip(SHAPES[1:], outs[1:]):
        assert np.array_equal(o, outs[0]), s


DEGENERATE = RAGGED + [
    (1, 9, (Side("periodic"),) * 4),
    (9, 1, (Side("periodic"),) * 4),
    (70, 1, (Side("outflow"), Side("outflow"), Side("periodic"), Side("periodic"))),
    (1, 70, (Side("periodic"), Side("periodic"), Side("outflow"), Side("reflect"))),
]


@pytest.mark.parametrize("nx,ny,sides", DEGENERATE)
def test_fp32_every_launch_shape_on_tiny_and_ragged_grids(nx, ny, sides):
    """Grids of one node, one row or one column, and grids smaller than a
    tile, with every boundary kind: every FP32 launch shape gives the same
    bits, and the tile kernel stays within FP32 accuracy of the FP64
    oracle."""
    rng = np.random.Generator(np.random.PCG64(nx * 1000 + ny + 7))
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), dx=0.01, alpha=0.1, sides=sides, steps=40)
    p = p.with_(tau=p.dt / 0.7)
    fields = (1.0 + 0.3 * rng.random((ny, nx)), 0.5 * rng.standard_normal((ny, nx)),
              0.5 * rng.standard_normal((ny, nx)), 1.0 + 0.3 * rng.random((ny, nx)))
    outs = []
    for shape in SHAPES:
        with lbm.Lattice(p, "fp32_cons") as lat:
            lbm.lbm_set_launch(lat.ctx, *shape)
            lat.init(*fields).step(p.steps)
            lat.sync()
            outs.append(lat.get_f().cpu().numpy())
    for shape, o in zip(SHAPES[1:], outs[1:]):
        assert np.array_equal(o, outs[0]), shape
    ref = oracle_run(p, fields=fields)[0]
    err = max_rel(gpu_run(p, "fp32_cons", fields=fields), ref)
    assert max(err.values()) <= 1e-4, err


@pytest.mark.parametrize("shape", [(3, 0, 0, 0), (1, 128, 4, 0), (2, 4, 0, 0), (2, 2, 0, 0)])
def test_fp32_kernels_match_oracle_on_ragged_grid(shape):
    p = W.dmr(37).with_(nx=151, steps=120)
    ref = cached_oracle("dmr151x37", p)
    with lbm.Lattice(p, "fp32") as lat:
        lbm.lbm_set_launch(lat.ctx, *shape)
        lat.init(*W.initial_fields(p)).step(p.steps)
        g = [t.double().cpu().numpy() for t in lat.moments()]
    assert l1_rel(g[0], ref[0]) <= 1e-4 and l1_rel(g[3], ref[3]) <= 1e-4


def test_autotune_restores_state_and_picks_a_shape():
    p = W.dmr(64)
    with lbm.Lattice(p, "fp32") as lat:
        lat.init(*W.initial_fields(p)).step(10)
        before = lat.get_f().cpu().numpy()
        best, ms = lbm.lbm_autotune(lat.ctx, 5)
        assert lat.step_count == 10
        assert np.array_equal(lat.get_f().cpu().numpy(), before)
        assert len(ms) == 7 and all(m > 0 for m in ms)
        assert lbm.lbm_get_launch(lat.ctx) == best
    with lbm.Lattice(p, "fp64") as lat:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_launch(lat.ctx, 1, 256, 4, 0)


def test_probe_tile_copy_measures_a_plausible_bandwidth():
    """The step kernel's data movement alone on the 4096 x 1024 grid and on a
    ragged one: a finite positive rate, below twice the device's nominal HBM
    bandwidth (it moves 72 bytes per node between HBM and the SMs)."""
    for nx, ny in ((4096, 1024), (333, 77)):
        g = lbm.lbm_probe_tile_copy(nx, ny, 3)
        assert np.isfinite(g) and 0.0 < g < 16000.0, (nx, ny, g)


def _bump_fields(p, cx, cy):
    """Uniform state with a smooth bump centred at node (cx, cy), built on the
    device: every value depends only on the offset from the centre, and the
    bump is exactly zero beyond about 30 nodes."""
    import torch
    y = torch.arange(p.ny, device="cuda", dtype=torch.float32)[:, None]
    x = torch.arange(p.nx, device="cuda", dtype=torch.float32)[None, :]
    g = torch.exp(-((x - cx) ** 2 + (y - cy) ** 2) / 8.0)
    one = torch.ones_like(g)
    return 1.0 + 0.05 * g, 0.1 * one, 0.05 * one, 1.0 + 0.02 * g


@pytest.mark.parametrize("variant", [3, 0])
def test_grid_past_2_31_elements_matches_a_small_grid(variant):
    """32768 x 8192 in FP32: a level holds 2.4e9 elements, past what 32-bit
    offsets can address.  A uniform periodic state with one smooth bump near
    the far corner evolves node for node like the same bump in the middle of
    a small periodic grid (the same update at every node; the disturbance
    spreads one node per step and never meets a boundary), so after a few
    steps the two windows around the bump agree bit for bit -- through the
    tile kernel and through the thread-per-node kernel."""
    import torch
    per = W.Side("periodic")
    st = (1.0, 0.1, 0.05, 1.0)
    big = W.uniform(32768, 8192, st, sides=(per,) * 4)
    small = W.uniform(256, 128, st, sides=(per,) * 4)
    n, h = 6, 40
    cx, cy = big.nx - 48, big.ny - 48
    with lbm.Lattice(big, "fp32_cons") as lat:
        lbm.lbm_set_launch(lat.ctx, variant)
        lat.init(*_bump_fields(big, cx, cy)).step(n)
        lat.sync()
        got = lat.get_f()[:, cy - h:cy + h, cx - h:cx + h].cpu().numpy()
    torch.cuda.empty_cache()
    with lbm.Lattice(small, "fp32_cons") as lat:
        lbm.lbm_set_launch(lat.ctx, variant)
        lat.init(*_bump_fields(small, 128, 64)).step(n)
        lat.sync()
        want = lat.get_f()[:, 64 - h:64 + h, 128 - h:128 + h].cpu().numpy()
    assert np.array_equal(got, want)
    assert np.max(np.abs(want - want[:, :1, :1])) > 1e-4  # the bump is there
