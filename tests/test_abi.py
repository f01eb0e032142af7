"""Host-side checks of the C ABI (no GPU compute): the library loads, exports
every entry point include/lbm.h declares, and rejects invalid arguments with
LBM_E_INVAL before touching the device."""
import math
import os
import re
import subprocess

import pytest

from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = lbm.load()
    declared = _declared()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.library_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (lbm_[a-z0-9_]+)$", out, flags=re.M))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lib, name)
    assert set(lbm.EXPORTS) <= declared


def test_library_is_built_for_sm103a():
    from paper_0706_0405_gb300 import build as B
    assert "arch=compute_103a,code=sm_103a" in B.ARCH


def _args(p, **over):
    dvm = lbm.lbm_dvm(over.get("c1", p.c1), over.get("c2", p.c2), over.get("eta0", p.eta0))
    diss = lbm.lbm_dissipation()
    diss.beta = over.get("beta", p.beta)
    lam = over.get("lam", p.lam)
    for i in range(9):
        diss.lambda_[i] = lam[i]
    sides = over.get("sides", p.sides)
    return (over.get("nx", p.nx), over.get("ny", p.ny), over.get("b", p.b), over.get("tau", p.tau),
            over.get("dt", p.dt), over.get("dx", p.dx), dvm, diss, [lbm.make_bc(s) for s in sides],
            over.get("prec", 0))


@pytest.mark.parametrize("over,msg", [
    ({"nx": 0}, "nx and ny"), ({"ny": -3}, "nx and ny"), ({"b": 0.0}, "b must"),
    ({"tau": -1.0}, "tau"), ({"dt": math.nan}, "dt"), ({"dx": 0.0}, "dx"),
    ({"c1": 9.0}, "singular"), ({"eta0": 0.0}, "eta0"), ({"beta": 0.6}, "beta"),
    ({"beta": -0.1}, "beta"), ({"lam": (0.1,) * 8 + (-1.0,)}, "lambda[8]"), ({"prec": 7}, "precision"),
    ({"sides": (W.Side("periodic"), W.Side("outflow"), W.Side("periodic"), W.Side("periodic"))},
     "periodic"),
    ({"sides": (W.Side("outflow"),) * 3 + (W.Side("dirichlet", state_lo=(-1.0, 0, 0, 1.0)),)},
     "Dirichlet"),
])
def test_create_rejects_invalid_arguments(over, msg):
    p = W.sod_400x4()
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(*_args(p, **over))
    assert ei.value.status == lbm.LBM_E_INVAL
    assert msg in str(ei.value)


def test_level_bytes_is_the_padded_row_interleaved_level():
    # (ny + 2) rows x 9 populations x pitch, pitch = nx + 8 rounded up to 32
    assert lbm.lbm_level_bytes(400, 4, "fp64") == 6 * 9 * 416 * 8
    assert lbm.lbm_level_bytes(400, 4, "fp32_tdf") == 6 * 9 * 416 * 4
    assert lbm.lbm_level_bytes(4096, 1024, "fp32") == 1026 * 9 * 4128 * 4
    assert lbm.lbm_level_bytes(1, 1, "fp32") == 3 * 9 * 32 * 4
    for bad in ((0, 4, "fp64"), (4, -1, "fp64"), (1 << 25, 4, "fp32"), (4, 4, 9)):
        assert lbm.lbm_level_bytes(*bad) == 0


@pytest.mark.parametrize("bufs,msg", [
    ((1 << 20, None), "both"), ((None, 1 << 20), "both"),
    (((1 << 20) + 16, 1 << 24), "aligned"), ((1 << 20, (1 << 20) + 256), "overlap"),
])
def test_create_rejects_bad_caller_buffers_before_touching_them(bufs, msg):
    # rejected by the argument checks alone: the addresses are never used
    p = W.sod_400x4()
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(*_args(p), None, *bufs)
    assert ei.value.status == lbm.LBM_E_INVAL
    assert msg in str(ei.value)


def test_calls_on_null_context_fail_cleanly():
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step(None, 1)
    assert ei.value.status == lbm.LBM_E_INVAL
    assert lbm.lbm_step_count(None) == -1
    assert lbm.lbm_checkpoint_bytes(None) == 0
    lbm.lbm_destroy(None)


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(*_args(W.sod_400x4()))
    assert ei.value.status in (lbm.LBM_E_CUDA, lbm.LBM_E_NOMEM)


def _vn(**over):
    p = W.sod_400x4()
    q = lbm.vn_case(p, over.pop("state", (1.0, 0.0, 0.0, 1.0)))
    for k, v in over.items():
        if k in ("c1", "c2", "eta0"):
            setattr(q.dvm, k, v)
        elif k == "beta":
            q.diss.beta = v
        elif k == "lam8":
            q.diss.lambda_[8] = v
        else:
            setattr(q, k, v)
    return q


@pytest.mark.parametrize("kw,msg", [
    (dict(cases=[_vn(c2=3.0)]), "case 0: c1"), (dict(cases=[_vn(), _vn(beta=0.7)]), "case 1: beta"),
    (dict(cases=[_vn(lam8=-1.0)]), "lambda[8]"), (dict(cases=[_vn(state=(1.0, 0.0, 0.0, 0.0))]), "T > 0"),
    (dict(cases=[_vn(tau=0.0)]), "tau"), (dict(dirs=[(0, 0)]), "direction 0"),
    (dict(dirs=[(1, 0)] * 65), "ndirs"), (dict(nk=0), "nk"), (dict(nk=70000), "nk"),
    (dict(growth=None), "both NULL"),
])
def test_vn_scan_rejects_invalid_arguments(kw, msg):
    import numpy as np
    args = dict(cases=[_vn()], dirs=[(1, 0)], nk=31, growth=np.zeros(1))
    args.update(kw)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_vn_scan(args["cases"], args["dirs"], args["nk"], growth=args["growth"])
    assert ei.value.status == lbm.LBM_E_INVAL
    assert msg in str(ei.value)


def test_vn_scan_with_no_cases_does_nothing():
    lbm.lbm_vn_scan([], [(1, 0)], 31)


@pytest.mark.parametrize("args", [(0, 8, 1), (8, 0, 1), (8, 8, 0)])
def test_probe_tile_copy_rejects_invalid_arguments(args):
    import ctypes
    g = ctypes.c_double(-1.0)
    assert lbm.load().lbm_probe_tile_copy(*args, ctypes.byref(g)) == lbm.LBM_E_INVAL
    assert lbm.load().lbm_probe_tile_copy(8, 8, 1, None) == lbm.LBM_E_INVAL
    assert g.value == -1.0


@pytest.mark.parametrize("seconds", [0.0, -1.0, float("nan"), 61.0])
def test_batch_wait_limit_rejects_out_of_range(seconds):
    assert lbm.load().lbm_batch_set_wait_limit(seconds) == lbm.LBM_E_INVAL


def test_batch_plant_stall_on_null_batch_fails_cleanly():
    assert lbm.load().lbm_batch_plant_stall(None, 0) == lbm.LBM_E_INVAL
