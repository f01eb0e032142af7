"""Failure detection on the GPU with failures made on the host: device
allocations that fail (lbm_inject_alloc_failure) must surface as
LBM_E_NOMEM from the call that needed them, free what that call had
allocated, and leave the library usable.  (Bounded device waits that run
out are covered by the batch tests; non-physical states by the parity
tests.)"""
import numpy as np
import pytest

from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def _each_failure(run, limit):
    """Run `run()` with the k-th device allocation failing, k = 0, 1, ...,
    until it succeeds; returns the number of runs that failed (each must
    fail with LBM_E_NOMEM)."""
    failed = 0
    for k in range(limit):
        lbm.lbm_inject_alloc_failure(k)
        try:
            run()
        except lbm.LbmError as e:
            assert e.status == lbm.LBM_E_NOMEM, (k, str(e))
            failed += 1
            continue
        finally:
            lbm.lbm_inject_alloc_failure(-1)
        return failed
    raise AssertionError(f"still failing after {limit} injected failures")


def test_injected_allocation_failures_surface_as_nomem_and_leak_nothing():
    st = (1.0, 0.1, 0.0, 1.0)
    p = W.uniform(130, 20, st, sides=(W.Side("outflow"),) * 2 + (W.Side("periodic"),) * 2)
    fields = W.initial_fields(p, seed=1, sigma=0.01)
    probs = [W.uniform(90, 4, st, sides=(W.Side("outflow"),) * 2 + (W.Side("periodic"),) * 2),
             W.uniform(200, 4, st, sides=(W.Side("outflow"),) * 2 + (W.Side("periodic"),) * 2)]
    bfields = [W.initial_fields(q, seed=2 + k, sigma=0.01) for k, q in enumerate(probs)]
    free0 = _free_bytes()

    def create():
        lbm.Lattice(p, "fp32_cons").close()

    def adjoint():
        with lbm.Lattice(p, "fp32_cons") as lat:
            lat.init(*fields)
            lbm.lbm_record(lat.ctx, 5)
            lat.step(10)
            abar = np.ones((9, p.ny, p.nx), np.float32)
            lbm.lbm_adjoint_step(lat.ctx, 10, abar)

    def batch():
        with lbm.Batch(probs, "fp32_cons") as b:
            b.init(bfields).step(5)
            b.sync()

    try:
        n_create = _each_failure(create, 40)
        n_adjoint = _each_failure(adjoint, 200)
        n_batch = _each_failure(batch, 200)
    finally:
        lbm.lbm_inject_alloc_failure(-1)
    # lbm_create makes five device allocations; the adjoint run and the batch
    # make more (checkpoints, adjoint and segment levels; one context per
    # problem, tables, counters)
    assert n_create == 5
    assert n_adjoint > n_create and n_batch > 2 * n_create
    # after all of that the device holds what it held before (allocation
    # granularity aside), and the library still works
    assert abs(_free_bytes() - free0) <= (32 << 20)
    with lbm.Lattice(p, "fp32_cons") as lat:
        lat.init(*fields).step(3)
        lat.sync()
