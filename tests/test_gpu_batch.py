"""The batched persistent launch (lbm_batch_*) against stepping each problem
alone and against the oracle."""
import numpy as np
import pytest

import oracle
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _subset():
    probs = W.batch_riemann()
    idx = [0, 3, 17, 42, 99, 128, 200, 255]
    return [probs[k] for k in idx]


@pytest.mark.parametrize("prec", ["fp32", "fp32_tdf", "fp32_cons"])
def test_batch_equals_problems_stepped_alone(prec):
    probs = _subset()
    fields = [W.initial_fields(p) for p in probs]
    with lbm.Batch(probs, prec) as b:
        b.init(fields).step(150).step(50)
        b.sync()
        grid, ntiles, graph = b.info()
        got = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    assert graph == 1 and ntiles > len(probs) and grid > 0
    for p, fl, g in zip(probs, fields, got):
        with lbm.Lattice(p, prec) as lat:
            lat.init(*fl).step(200)
            want = lat.get_f().cpu().numpy()
        assert np.array_equal(g, want), p.name


def test_batch_matches_oracle():
    probs = W.batch_riemann()
    pick = [5, 77, 180]
    with lbm.Batch(probs, "fp32") as b:
        b.init([W.initial_fields(p) for p in probs]).step(1000)
        b.sync()
        got = {k: [t.double().cpu().numpy() for t in b.moments(k)] for k in pick}
    oracle.set_threads(oracle.max_threads())
    for k in pick:
        p = probs[k]
        f = oracle.init(p, *W.initial_fields(p))
        assert oracle.run(p, f, 1000) == 0
        ref = oracle.fields(p, f)
        for q in (0, 3):
            l1 = np.sum(np.abs(got[k][q] - ref[q])) / np.sum(np.abs(ref[q]))
            assert l1 <= 1e-3, (p.name, q, l1)


def test_batch_argument_errors():
    probs = _subset()[:2]
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Batch(probs, "fp64")
    assert ei.value.status == lbm.LBM_E_INVAL
    with lbm.Batch(probs, "fp32") as b:
        with pytest.raises(lbm.LbmError) as ei:
            b.step(1)
        assert ei.value.status == lbm.LBM_E_STATE


@pytest.mark.parametrize("shape", [(2, 0, 0), (1, 7, 0), (2, 3, 0), (1, 0, 3), (1, 0, 5), (1, 5, 7)])
def test_every_batch_launch_shape_gives_the_same_bits(shape):
    """Two nodes per thread (128-thread CTAs), grids of a few CTAs, and
    temporal blocking with 3, 5 or 7 steps per pass (120 steps: whole passes
    and a shorter last one) do the same per-node arithmetic and ghost rules:
    the levels equal those of the default shape (one node per thread, one
    step per launch pass, a full wave) bit for bit."""
    probs = _subset()
    fields = [W.initial_fields(p) for p in probs]
    out = {}
    for sh in [(1, 0, 0), shape]:
        with lbm.Batch(probs, "fp32_cons") as b:
            b.init(fields).set_launch(*sh).step(120)
            b.sync()
            out[sh] = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    for a, c in zip(out[(1, 0, 0)], out[shape]):
        assert np.array_equal(a, c)


def test_batch_autotune_restores_state_and_picks_a_shape():
    probs = _subset()
    fields = [W.initial_fields(p) for p in probs]
    with lbm.Batch(probs, "fp32_cons") as b:
        b.init(fields).step(30)
        (npt, grid, block), ms = b.autotune(steps=5)
        assert len(ms) == 7 and all(m > 0 for m in ms)
        assert (npt, grid, block) == b.get_launch() and npt in (1, 2) and grid > 0 and block in (0, 3, 5, 7)
        b.step(40)
        b.sync()
        grid_info, _, graph = b.info()
        got = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    assert graph == 1 and grid_info == grid
    with lbm.Batch(probs, "fp32_cons") as b:
        b.init(fields).step(70)
        b.sync()
        want = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    for a, c in zip(got, want):
        assert np.array_equal(a, c)


def test_batch_launch_shape_errors():
    probs = _subset()[:2]
    with lbm.Batch(probs, "fp32") as b:
        for bad in [(3, 0, 0), (1, -1, 0), (2, 10 ** 6, 0), (1, 0, 4), (1, 10 ** 6, 3)]:
            with pytest.raises(lbm.LbmError) as ei:
                b.set_launch(*bad)
            assert ei.value.status == lbm.LBM_E_INVAL
    wide = [W.uniform(70, 12, (1.0, 0.1, 0.0, 1.0), sides=(W.Side("outflow"),) * 4)]
    with lbm.Batch(wide, "fp32") as b:  # 12 rows: too many for temporal blocking
        with pytest.raises(lbm.LbmError) as ei:
            b.set_launch(1, 0, 3)
        assert ei.value.status == lbm.LBM_E_INVAL


def _mixed():
    """Problems of 1 to 9 rows with perturbed fields: periodic in y with the
    whole height inside one tile row (1 to 4 rows), periodic in y over two
    tile rows (9 rows), periodic in x and y, reflecting walls."""
    P, O, R = W.Side("periodic"), W.Side("outflow"), W.Side("reflect")
    st = (1.0, 0.1, 0.05, 1.0)
    return [W.uniform(100, 1, st, sides=(O, O, P, P)), W.uniform(70, 2, st, sides=(P, P, P, P)),
            W.uniform(130, 3, st, sides=(O, O, P, P)), W.uniform(64, 4, st, sides=(P, P, P, P)),
            W.uniform(90, 9, st, sides=(O, O, P, P)), W.uniform(50, 5, st, sides=(O, O, R, R)),
            W.uniform(200, 4, st, sides=(O, O, P, P))]


@pytest.mark.parametrize("shape", [(1, 0, 0), (2, 0, 0), (1, 3, 0), (2, 2, 0)])
def test_mixed_heights_and_sides_equal_problems_stepped_alone(shape):
    """Heights 1 to 9 and every y rule: problems whose tile holds every row
    take their periodic y neighbours from the tile and write their y ghost
    rows on a launch's last step only; over several calls of several steps
    the levels equal those of each problem stepped alone, bit for bit."""
    probs = _mixed()
    fields = [W.initial_fields(p, seed=k, sigma=0.01) for k, p in enumerate(probs)]
    with lbm.Batch(probs, "fp32_cons") as b:
        b.init(fields).set_launch(*shape).step(25).step(1).step(34)
        b.sync()
        got = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    for p, fl, g in zip(probs, fields, got):
        with lbm.Lattice(p, "fp32_cons") as lat:
            lat.init(*fl).step(60)
            want = lat.get_f().cpu().numpy()
        assert np.array_equal(g, want), p.name


def test_switching_to_temporal_blocking_mid_run_keeps_the_bits():
    """The tile kernel leaves the level with valid ghost rows at the end of
    every launch, so the temporal-blocking kernel (which reads them) can take
    over between calls."""
    probs = _subset()
    fields = [W.initial_fields(p) for p in probs]
    with lbm.Batch(probs, "fp32_cons") as b:
        b.init(fields).step(50).set_launch(1, 0, 3).step(50).set_launch(2, 0, 0).step(20)
        b.sync()
        got = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    for p, fl, g in zip(probs, fields, got):
        with lbm.Lattice(p, "fp32_cons") as lat:
            lat.init(*fl).step(120)
            want = lat.get_f().cpu().numpy()
        assert np.array_equal(g, want), p.name


def test_a_neighbour_that_never_finishes_times_out_and_the_batch_recovers():
    """Failure injected on the host: one CTA is told to wait for a counter no
    CTA advances.  Its bounded wait runs out (0.2 s here), the launch stops,
    LBM_E_TIMEOUT reaches the caller, and after lbm_batch_init the same batch
    steps correctly again (bit for bit against each problem alone)."""
    probs = _subset()
    fields = [W.initial_fields(p) for p in probs]
    lbm.lbm_batch_set_wait_limit(0.2)
    try:
        with lbm.Batch(probs, "fp32_cons") as b:
            b.set_launch(1, 0, 0).init(fields).step(3)
            b.sync()
            b.plant_stall(1)
            with pytest.raises(lbm.LbmError) as ei:
                b.step(6)
                b.sync()
            assert ei.value.status == lbm.LBM_E_TIMEOUT
            b.plant_stall(-1)
            b.init(fields).step(10)
            b.sync()
            got = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    finally:
        lbm.lbm_batch_set_wait_limit(2.0)
    for p, fl, g in zip(probs, fields, got):
        with lbm.Lattice(p, "fp32_cons") as lat:
            lat.init(*fl).step(10)
            want = lat.get_f().cpu().numpy()
        assert np.array_equal(g, want), p.name


def test_one_column_and_one_node_problems_in_a_batch():
    """Problems one node wide, one node in all, and a few nodes in each
    direction, periodic or not, stepped together: each equals the problem
    stepped alone, bit for bit."""
    P, O, R = W.Side("periodic"), W.Side("outflow"), W.Side("reflect")
    st = (1.0, 0.1, 0.05, 1.0)
    probs = [W.uniform(1, 1, st, sides=(P, P, P, P)), W.uniform(1, 6, st, sides=(P, P, O, R)),
             W.uniform(2, 2, st, sides=(O, O, P, P)), W.uniform(3, 5, st, sides=(R, R, R, R)),
             W.uniform(65, 4, st, sides=(O, O, P, P))]
    fields = [W.initial_fields(p, seed=10 + k, sigma=0.01) for k, p in enumerate(probs)]
    with lbm.Batch(probs, "fp32_cons") as b:
        b.init(fields).step(17).step(13)
        b.sync()
        got = [b.get_f(k).cpu().numpy() for k in range(len(probs))]
    for p, fl, g in zip(probs, fields, got):
        with lbm.Lattice(p, "fp32_cons") as lat:
            lat.init(*fl).step(30)
            want = lat.get_f().cpu().numpy()
        assert np.array_equal(g, want), p.name
