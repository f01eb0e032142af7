"""Caller-owned level buffers (lbm_create's f_buf0 / f_buf1): the state f of
Eq. (SEC-VON-1) stepped in memory the caller allocated (here: slices of one
torch CUDA tensor), bit for bit as in library-owned buffers, and left alive
and untouched when the context is destroyed."""
import numpy as np
import pytest
import torch

from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _carve(nbytes):
    """Two 256-byte aligned, non-overlapping slices of one uint8 CUDA tensor,
    neither at the start of the tensor's allocation; returns (pool, b0, b1)."""
    span = (nbytes + 255) // 256 * 256
    pool = torch.zeros(2 * span + 1024, dtype=torch.uint8, device="cuda")
    off0 = (-pool.data_ptr()) % 256 + 256
    off1 = off0 + span
    return pool, pool[off0:off0 + nbytes], pool[off1:off1 + nbytes]


def _interior(buf, p, prec):
    """The 9 x ny x nx interior of a level in the library's layout: row
    iy + 1, the nine population rows of a grid row together, column ix + 4."""
    dt = torch.float64 if prec == "fp64" else torch.float32
    pitch = (p.nx + 8 + 31) // 32 * 32
    a = buf.view(dt).view(p.ny + 2, 9, pitch)
    return a[1:p.ny + 1, :, 4:4 + p.nx].permute(1, 0, 2).contiguous()


@pytest.mark.parametrize("prec", ["fp64", "fp32_tdf", "fp32_cons"])
def test_caller_owned_buffers_give_the_same_bits_and_outlive_the_context(prec):
    p = W.dmr(64)  # 256 x 64, every boundary kind, a moving split on the top
    steps = 41     # odd: the current level ends in the second buffer
    fields = W.initial_fields(p)
    nbytes = lbm.Lattice.level_bytes(p, prec)
    pool, b0, b1 = _carve(nbytes)
    guard = pool.clone()
    with lbm.Lattice(p, prec, buffers=(b0, b1)) as lat:
        lat.init(*fields).step(steps)
        lat.sync()
        got = lat.get_f()
        held = _interior((b0, b1)[steps % 2], p, prec)
    with lbm.Lattice(p, prec) as ref:
        ref.init(*fields).step(steps)
        want = ref.get_f()
    assert torch.equal(got, want)
    # the current level lives in the caller's memory
    assert torch.equal(held, want)
    # destroying the context neither freed nor wrote the caller's tensors
    torch.cuda.synchronize()
    after = pool.clone()
    assert torch.equal(_interior((b0, b1)[steps % 2], p, prec), want)
    assert torch.equal(after[:256], guard[:256])  # bytes before the first buffer untouched
    pool.add_(1)  # still a live allocation the caller can use
    torch.cuda.synchronize()
    assert torch.equal(pool, after + 1)


def test_caller_buffers_must_be_device_memory_of_this_device():
    p = W.sod_400x4()
    nbytes = lbm.Lattice.level_bytes(p, "fp64")
    host = [np.zeros(nbytes + 256, dtype=np.uint8) for _ in range(2)]
    ptrs = [h.ctypes.data + (-h.ctypes.data) % 256 for h in host]
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice(p, "fp64", buffers=ptrs)
    assert ei.value.status == lbm.LBM_E_INVAL
    assert "device memory" in str(ei.value)
    # too small a gap between the two buffers
    pool, b0, _ = _carve(nbytes)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice(p, "fp64", buffers=(b0.data_ptr(), b0.data_ptr() + 256))
    assert ei.value.status == lbm.LBM_E_INVAL
    del pool


def test_caller_buffers_serve_the_adjoint_and_checkpoints():
    # the recorded checkpoints and the adjoint's recomputation read the
    # levels through the same pointers
    # a small Mach-3 tube: (rho, ux, uy, p) left and right
    q = W.riemann("mach3_small", 256, 8, 1.0, (1.4, 3.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0), 0.5,
                  4.0, 10.0, 6.0, alpha=0.05, steps=30)
    fields = W.initial_fields(q, seed=0, sigma=0.01)
    res = []
    for owned in (True, False):
        pool = None
        bufs = None
        if not owned:
            pool, b0, b1 = _carve(lbm.Lattice.level_bytes(q, "fp32_tdf"))
            bufs = (b0, b1)
        with lbm.Lattice(q, "fp32_tdf", buffers=bufs) as la:
            la.init(*fields)
            lbm.lbm_record(la.ctx, 10)
            la.step(q.steps)
            abar = torch.zeros((9, q.ny, q.nx), dtype=la.dtype, device="cuda")
            lbm.lbm_adjoint_seed(la.ctx, torch.ones((q.ny, q.nx), dtype=la.dtype, device="cuda"), None, None,
                                 None, abar)
            dtau = lbm.lbm_adjoint_step(la.ctx, q.steps, abar)
            res.append((abar.cpu(), dtau))
        del pool
    assert torch.equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
