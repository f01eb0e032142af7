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
