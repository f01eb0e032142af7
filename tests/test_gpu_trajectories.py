"""Whole trajectories against the FP64 oracle, in every precision mode:

  * the double Mach reflection (Sec. 4.2, Fig. 12) at 1024 x 256 to t = 0.2,
    10 240 steps, the same geometry and boundary kinds as the 4096 x 1024
    benchmark grid;
  * all 256 tubes of the batched Riemann sweep for their 1 000 steps, run
    together in one persistent launch, including the 61 that pass through
    T < 0 behind their shocks.

Bars (the error measures of test_gpu_parity.py):
  * FP64: 1e-10 max relative error in rho, u, T;
  * FP32 modes: L1 relative error of rho and T <= 1e-3 across shocks,
    <= 1e-4 on smooth flow (the still gas ahead of the double Mach
    reflection's incident shock), shock position within one cell.
One stated exception: plain FP32 (no moment-exact relaxation) drifts in T
at high Mach, because the equilibrium built from FP32 moments does not
carry their energy, a bias that grows with u^2 / T.  Its T bar across the
sweep is 5e-2.  The moment-exact modes measure at most 1.3e-4 there.
"""
import numpy as np
import pytest

import oracle
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_MODES = ("fp32", "fp32_t64", "fp32_tdf", "fp32_cons")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(oracle.max_threads())
    yield
    oracle.set_threads(1)


def max_rel(g, r):
    rho = np.max(np.abs(g[0] - r[0]) / np.abs(r[0]))
    T = np.max(np.abs(g[3] - r[3]) / np.abs(r[3]))
    U = max(np.max(np.abs(r[1])), np.max(np.abs(r[2])), np.sqrt(np.max(r[3])))
    u = max(np.max(np.abs(g[1] - r[1])), np.max(np.abs(g[2] - r[2]))) / U
    return {"rho": rho, "u": u, "T": T}


def l1_rel(a, b):
    return float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))


# ------------------------------------------------ double Mach reflection

@pytest.fixture(scope="module")
def dmr_ref():
    p = W.dmr(256)
    assert p.steps == 10240
    f = oracle.init(p, *W.initial_fields(p))
    assert oracle.run(p, f, p.steps) == 0
    return p, oracle.fields(p, f)


def _dmr_gpu(p, prec):
    with lbm.Lattice(p, prec) as lat:
        lat.init(*W.initial_fields(p)).step(p.steps)
        return [t.double().cpu().numpy() for t in lat.moments()]


def _incident_shock_column(rho_row):
    """Rightmost cell of a row above the midpoint of the pre- and post-shock
    densities (1.4, 8): the incident shock, which runs into still gas."""
    return int(np.nonzero(rho_row > 0.5 * (1.4 + 8.0))[0].max())


def test_dmr_1024x256_full_run_fp64(dmr_ref):
    p, ref = dmr_ref
    err = max_rel(_dmr_gpu(p, "fp64"), ref)
    assert max(err.values()) <= 1e-10, err


@pytest.mark.parametrize("prec", FP32_MODES)
def test_dmr_1024x256_full_run_fp32_modes(dmr_ref, prec):
    p, ref = dmr_ref
    g = _dmr_gpu(p, prec)
    assert l1_rel(g[0], ref[0]) <= 1e-3 and l1_rel(g[3], ref[3]) <= 1e-3
    # smooth flow: the still gas ahead of the incident shock (all columns
    # more than 16 cells right of the shock in every row)
    ahead = np.zeros(ref[0].shape, dtype=bool)
    for row in range(p.ny):
        ahead[row, _incident_shock_column(ref[0][row]) + 16:] = True
    assert ahead.sum() > p.nodes // 4
    for q in (0, 3):
        assert l1_rel(g[q][ahead], ref[q][ahead]) <= 1e-4, (prec, q)
    for row in (16, 64, 128, 192, 240):
        assert abs(_incident_shock_column(g[0][row]) - _incident_shock_column(ref[0][row])) <= 1, (prec, row)


# ----------------------------------------------------- 256-tube batch

@pytest.fixture(scope="module")
def batch_ref():
    probs = W.batch_riemann()
    refs = []
    for q in probs:
        f = oracle.init(q, *W.initial_fields(q))
        oracle.run(q, f, q.steps)
        refs.append(oracle.fields(q, f))
    return probs, refs


def _shock_cell(rho_row):
    """Rightmost cell of a tube above 1.5 times the right state's density
    (1): the right-running shock, or -1 if the tube has none."""
    idx = np.nonzero(rho_row > 1.5)[0]
    return int(idx.max()) if len(idx) else -1


@pytest.mark.parametrize("prec", ["fp32_cons", "fp32_tdf", "fp32"])
def test_all_256_batch_tubes_match_the_oracle(batch_ref, prec):
    probs, refs = batch_ref
    with lbm.Batch(probs, prec) as b:
        b.init([W.initial_fields(q) for q in probs]).step(probs[0].steps)
        b.sync()
        got = [[t.double().cpu().numpy() for t in b.moments(k)] for k in range(len(probs))]
        t_neg = [bool(lbm.lbm_health(lbm.lbm_batch_problem(b.handle, k)) & lbm.LBM_FLAG_T_NONPOSITIVE)
                 for k in range(len(probs))]
    assert sum(t_neg) == 61  # the tubes that pass through T < 0, as in the oracle runs
    bar_T = 5e-2 if prec == "fp32" else 1e-3
    for q, g, r in zip(probs, got, refs):
        assert l1_rel(g[0], r[0]) <= 1e-3, (prec, q.name)
        assert abs(_shock_cell(g[0][0]) - _shock_cell(r[0][0])) <= 1, (prec, q.name)
        assert l1_rel(g[3], r[3]) <= bar_T, (prec, q.name, l1_rel(g[3], r[3]))
