"""lbm_conservation_noalloc: the conservation totals for callers that cannot
allocate device memory (their memory is committed to a fixed pool, or an
allocation could stall a latency-critical loop).  Its scratch is a fixed array
inside the library, so it must give the same totals as lbm_conservation, call
after call, without depending on what an earlier call left there.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dvm = lbm.lbm_dvm(10.0, 20.0, 15.0)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conservation_noalloc(1, 4096, 2049, "fp32", dvm)  # 8 392 704 > 8 388 608 nodes
    assert ei.value.status == lbm.LBM_E_INVAL
    # checked before any CUDA call: each gives LBM_E_INVAL, not LBM_E_CUDA
    for args in ((1, 0, 5, "fp32"), (1, 5, 0, "fp32"), (1, 5, 5, 9), (None, 5, 5, "fp32")):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_conservation_noalloc(*args, dvm)
        assert ei.value.status == lbm.LBM_E_INVAL, args


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_totals_equal_lbm_conservation_twice(prec):
    import torch
    p = W.dmr(64)
    dvm = lbm.lbm_dvm(p.c1, p.c2, p.eta0)
    stream = torch.cuda.current_stream().cuda_stream
    with lbm.Lattice(p, prec) as lat:
        lat.init(*W.initial_fields(p)).step(30)
        for extra in (0, 11):  # two calls in a row, on two different levels
            lat.step(extra)
            f = lat.get_f()
            want = lat.conservation()
            got = lbm.lbm_conservation_noalloc(f, p.nx, p.ny, prec, dvm, stream)
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * abs(want[0])), (extra, got, want)
        # a smaller grid after a larger one: the stale partials must not leak in
        q = W.dmr(16)
        with lbm.Lattice(q, prec) as small:
            small.init(*W.initial_fields(q)).step(5)
            fs = small.get_f()
            want = small.conservation()
            got = lbm.lbm_conservation_noalloc(fs, q.nx, q.ny, prec, lbm.lbm_dvm(q.c1, q.c2, q.eta0),
                                               stream)
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * abs(want[0]))
