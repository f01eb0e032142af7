"""ctypes binding of ``liblbm.so`` (C ABI in ``include/lbm.h``).

The module-level functions carry the C names and only marshal arguments:
pointers may be given as torch tensors, numpy arrays, integers or None.  All
computation runs in the CUDA library; there is no CPU path.  If the library
cannot be loaded, every call raises.

``Lattice`` wraps one context for a problem description (the attributes of
``workloads.Problem``) and converts results to numpy/torch.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

LBM_OK, LBM_E_INVAL, LBM_E_NOMEM, LBM_E_CUDA, LBM_E_NONPHYSICAL, LBM_E_TIMEOUT, LBM_E_STATE = \
    0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_E_INVAL", -2: "LBM_E_NOMEM", -3: "LBM_E_CUDA",
                -4: "LBM_E_NONPHYSICAL", -5: "LBM_E_TIMEOUT", -6: "LBM_E_STATE"}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_t64": 2, "fp32_tdf": 3, "fp32_cons": 4}
BC_KINDS = {"periodic": 0, "outflow": 1, "dirichlet": 2, "reflect": 3}

# Exported symbols of include/lbm.h.
EXPORTS = ("lbm_create", "lbm_destroy", "lbm_last_error", "lbm_init", "lbm_step", "lbm_moments",
           "lbm_conservation", "lbm_sync", "lbm_get_f", "lbm_set_f", "lbm_step_count",
           "lbm_checkpoint_bytes", "lbm_save", "lbm_load", "lbm_version", "lbm_health",
           "lbm_set_launch", "lbm_get_launch", "lbm_autotune", "lbm_conservation_noalloc",
           "lbm_record", "lbm_adjoint_seed", "lbm_adjoint_step", "lbm_feq_vjp",
           "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_init",
           "lbm_batch_step", "lbm_batch_sync", "lbm_batch_problem", "lbm_batch_info",
           "lbm_probe_rates", "lbm_vn_scan", "lbm_batch_set_launch", "lbm_batch_get_launch",
           "lbm_batch_autotune", "lbm_probe_tile_copy", "lbm_batch_set_wait_limit", "lbm_batch_plant_stall",
           "lbm_inject_alloc_failure", "lbm_level_bytes")
LBM_FLAG_NONPHYSICAL, LBM_FLAG_TIMEOUT, LBM_FLAG_T_NONPOSITIVE = 1, 2, 4


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lbm_bc(ctypes.Structure):
    _fields_ = [("kind_lo", ctypes.c_int), ("kind_hi", ctypes.c_int),
                ("split0", ctypes.c_double), ("split_speed", ctypes.c_double),
                ("state_lo", ctypes.c_double * 4), ("state_hi", ctypes.c_double * 4)]


class lbm_dvm(ctypes.Structure):
    _fields_ = [("c1", ctypes.c_double), ("c2", ctypes.c_double), ("eta0", ctypes.c_double)]


class lbm_dissipation(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("lambda_", ctypes.c_double * 9)]


class lbm_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("b", ctypes.c_double),
                ("tau", ctypes.c_double), ("dt", ctypes.c_double), ("dx", ctypes.c_double),
                ("dvm", lbm_dvm), ("diss", lbm_dissipation), ("bc", lbm_bc * 4)]


class lbm_batch_launch(ctypes.Structure):
    _fields_ = [("npt", ctypes.c_int), ("grid", ctypes.c_int), ("block", ctypes.c_int)]

    def as_tuple(self):
        return (self.npt, self.grid, self.block)


class lbm_vn_case(ctypes.Structure):
    _fields_ = [("b", ctypes.c_double), ("tau", ctypes.c_double), ("dt", ctypes.c_double),
                ("dx", ctypes.c_double), ("dvm", lbm_dvm), ("diss", lbm_dissipation),
                ("state", ctypes.c_double * 4)]


class lbm_launch(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tx", ctypes.c_int), ("ring", ctypes.c_int),
                ("grid", ctypes.c_int)]

    def as_tuple(self):
        return (self.variant, self.tx, self.ring, self.grid)


_lib = None
_VP = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load():
    """Open liblbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build_library() if _build.stale() else _build.LIB
    lib = ctypes.CDLL(path)
    ctx = _VP
    sig = {
        "lbm_create": ([ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 +
                       [ctypes.POINTER(lbm_dvm), ctypes.POINTER(lbm_dissipation),
                        ctypes.POINTER(lbm_bc), ctypes.c_int, _VP, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
        "lbm_level_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
        "lbm_destroy": ([ctx], None),
        "lbm_last_error": ([ctx], ctypes.c_char_p),
        "lbm_init": ([ctx, _VP, _VP, _VP, _VP], ctypes.c_int),
        "lbm_step": ([ctx, ctypes.c_int], ctypes.c_int),
        "lbm_moments": ([ctx, _VP, _VP, _VP, _VP], ctypes.c_int),
        "lbm_conservation": ([ctx, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "lbm_sync": ([ctx], ctypes.c_int),
        "lbm_health": ([ctx, ctypes.POINTER(ctypes.c_uint)], ctypes.c_int),
        "lbm_get_f": ([ctx, _VP], ctypes.c_int),
        "lbm_set_f": ([ctx, _VP, ctypes.c_longlong], ctypes.c_int),
        "lbm_step_count": ([ctx], ctypes.c_longlong),
        "lbm_checkpoint_bytes": ([ctx], ctypes.c_size_t),
        "lbm_save": ([ctx, _VP, ctypes.c_size_t], ctypes.c_int),
        "lbm_load": ([ctx, _VP, ctypes.c_size_t], ctypes.c_int),
        "lbm_version": ([], ctypes.c_char_p),
        "lbm_set_launch": ([ctx, ctypes.POINTER(lbm_launch)], ctypes.c_int),
        "lbm_record": ([ctx, ctypes.c_int], ctypes.c_int),
        "lbm_probe_rates": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
        "lbm_probe_tile_copy": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
                                ctypes.c_int),
        "lbm_batch_set_wait_limit": ([ctypes.c_double], ctypes.c_int),
        "lbm_batch_plant_stall": ([_VP, ctypes.c_int], ctypes.c_int),
        "lbm_inject_alloc_failure": ([ctypes.c_longlong], ctypes.c_int),
        "lbm_batch_create": ([ctypes.c_int, ctypes.POINTER(lbm_problem), ctypes.c_int, _VP,
                              ctypes.POINTER(_VP)], ctypes.c_int),
        "lbm_batch_destroy": ([_VP], None),
        "lbm_batch_last_error": ([_VP], ctypes.c_char_p),
        "lbm_batch_init": ([_VP] + [ctypes.POINTER(_VP)] * 4, ctypes.c_int),
        "lbm_batch_step": ([_VP, ctypes.c_int], ctypes.c_int),
        "lbm_batch_sync": ([_VP], ctypes.c_int),
        "lbm_batch_problem": ([_VP, ctypes.c_int], _VP),
        "lbm_batch_info": ([_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "lbm_adjoint_seed": ([ctx, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "lbm_adjoint_step": ([ctx, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "lbm_feq_vjp": ([ctx] + [_VP] * 9, ctypes.c_int),
        "lbm_conservation_noalloc": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(lbm_dvm), ctypes.POINTER(ctypes.c_double), _VP],
                                     ctypes.c_int),
        "lbm_get_launch": ([ctx, ctypes.POINTER(lbm_launch)], ctypes.c_int),
        "lbm_batch_set_launch": ([_VP, ctypes.POINTER(lbm_batch_launch)], ctypes.c_int),
        "lbm_batch_get_launch": ([_VP, ctypes.POINTER(lbm_batch_launch)], ctypes.c_int),
        "lbm_batch_autotune": ([_VP, ctypes.c_int, ctypes.POINTER(lbm_batch_launch), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "lbm_vn_scan": ([ctypes.POINTER(lbm_vn_case), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                         ctypes.c_int, _VP, _VP, _VP], ctypes.c_int),
        "lbm_autotune": ([ctx, ctypes.c_int, ctypes.POINTER(lbm_launch),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(x):
    """Address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to liblbm must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays passed to liblbm must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x).__name__} as a pointer")


def _check(ctx, status):
    if status != LBM_OK:
        raise LbmError(status, load().lbm_last_error(ctx).decode())
    return status


# ------------------------------------------------------------- C-ABI calls

def lbm_version() -> str:
    return load().lbm_version().decode()


def _prec(prec) -> int:
    return PRECISIONS.get(prec, prec) if isinstance(prec, str) else int(prec)


def lbm_level_bytes(nx, ny, prec) -> int:
    """Bytes of one level buffer of a context (0 for invalid arguments)."""
    return int(load().lbm_level_bytes(int(nx), int(ny), _prec(prec)))


def lbm_create(nx, ny, b, tau, dt, dx, dvm, diss, bc, prec, stream=None, f_buf0=None, f_buf1=None):
    """Returns the context handle (int).  ``bc`` is a sequence of 4 lbm_bc;
    f_buf0 / f_buf1: optional caller-owned level buffers (device memory)."""
    lib = load()
    arr = (lbm_bc * 4)(*bc)
    out = _VP()
    st = lib.lbm_create(int(nx), int(ny), float(b), float(tau), float(dt), float(dx),
                        ctypes.byref(dvm), ctypes.byref(diss), arr, _prec(prec),
                        _ptr(stream), _ptr(f_buf0), _ptr(f_buf1), ctypes.byref(out))
    _check(None, st)
    return out.value


def lbm_destroy(ctx) -> None:
    load().lbm_destroy(ctx)


def lbm_last_error(ctx=None) -> str:
    return load().lbm_last_error(ctx).decode()


def lbm_init(ctx, rho, ux, uy, T):
    return _check(ctx, load().lbm_init(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T)))


def lbm_step(ctx, n):
    return _check(ctx, load().lbm_step(ctx, int(n)))


def lbm_moments(ctx, rho, ux, uy, T):
    return _check(ctx, load().lbm_moments(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T)))


def lbm_conservation(ctx):
    out = (ctypes.c_double * 4)()
    _check(ctx, load().lbm_conservation(ctx, out))
    return np.array(out[:])


def lbm_sync(ctx):
    return _check(ctx, load().lbm_sync(ctx))


def lbm_health(ctx) -> int:
    flags = ctypes.c_uint(0)
    _check(ctx, load().lbm_health(ctx, ctypes.byref(flags)))
    return int(flags.value)


def lbm_get_f(ctx, dst):
    return _check(ctx, load().lbm_get_f(ctx, _ptr(dst)))


def lbm_set_f(ctx, src, step=0):
    return _check(ctx, load().lbm_set_f(ctx, _ptr(src), int(step)))


def lbm_step_count(ctx) -> int:
    return int(load().lbm_step_count(ctx))


def lbm_checkpoint_bytes(ctx) -> int:
    return int(load().lbm_checkpoint_bytes(ctx))


def lbm_save(ctx, buf, nbytes):
    return _check(ctx, load().lbm_save(ctx, _ptr(buf), int(nbytes)))


def lbm_load(ctx, buf, nbytes):
    return _check(ctx, load().lbm_load(ctx, _ptr(buf), int(nbytes)))


def lbm_conservation_noalloc(f, nx, ny, prec, dvm, stream=None):
    """Totals of a dense 9 x ny x nx device distribution without allocating
    (see include/lbm.h); returns a numpy array of 4 doubles."""
    out = (ctypes.c_double * 4)()
    st = load().lbm_conservation_noalloc(
        _ptr(f), int(nx), int(ny), PRECISIONS.get(prec, prec) if isinstance(prec, str) else int(prec),
        ctypes.byref(dvm), out, _ptr(stream))
    if st != LBM_OK:
        raise LbmError(st, "lbm_conservation_noalloc failed")
    return np.array(out[:])


def lbm_record(ctx, every):
    return _check(ctx, load().lbm_record(ctx, int(every)))


def lbm_adjoint_seed(ctx, qr, qx, qy, qT, abar):
    return _check(ctx, load().lbm_adjoint_seed(ctx, _ptr(qr), _ptr(qx), _ptr(qy), _ptr(qT), _ptr(abar)))


def lbm_adjoint_step(ctx, n, abar):
    """Returns the tau derivative of the n steps."""
    d = ctypes.c_double(0.0)
    _check(ctx, load().lbm_adjoint_step(ctx, int(n), _ptr(abar), ctypes.byref(d)))
    return float(d.value)


def lbm_feq_vjp(ctx, rho, ux, uy, T, abar, g_rho, g_ux, g_uy, g_T):
    return _check(ctx, load().lbm_feq_vjp(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T), _ptr(abar),
                                          _ptr(g_rho), _ptr(g_ux), _ptr(g_uy), _ptr(g_T)))


def lbm_set_launch(ctx, variant, tx=256, ring=4, grid=0):
    return _check(ctx, load().lbm_set_launch(ctx, ctypes.byref(lbm_launch(variant, tx, ring, grid))))


def lbm_get_launch(ctx):
    out = lbm_launch()
    _check(ctx, load().lbm_get_launch(ctx, ctypes.byref(out)))
    return out.as_tuple()


def lbm_autotune(ctx, steps=20):
    """Returns (chosen (variant, tx, ring, grid), per-candidate ms per step)."""
    best = lbm_launch()
    ms = (ctypes.c_double * 8)()
    n = ctypes.c_int(0)
    _check(ctx, load().lbm_autotune(ctx, int(steps), ctypes.byref(best), ms, ctypes.byref(n)))
    return best.as_tuple(), list(ms[: n.value])


def lbm_probe_rates():
    """(FP64 TFLOP/s, FP32 TFLOP/s) of the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().lbm_probe_rates(ctypes.byref(a), ctypes.byref(b))
    if st != LBM_OK:
        raise LbmError(st, "lbm_probe_rates failed")
    return a.value, b.value


def lbm_probe_tile_copy(nx: int, ny: int, reps: int = 10) -> float:
    """GB/s (72 bytes per node) of the FP32 tile step's data movement alone on
    an nx x ny grid."""
    g = ctypes.c_double()
    st = load().lbm_probe_tile_copy(int(nx), int(ny), int(reps), ctypes.byref(g))
    if st != LBM_OK:
        raise LbmError(st, "lbm_probe_tile_copy failed")
    return g.value


DIRECTIONS = ((1, 0), (0, 1), (1, 1), (1, -1))


def lbm_vn_scan(cases, dirs, nk, radius=None, growth=None, stream=None):
    """Spectral radius of the amplification matrix for every case (a sequence
    of lbm_vn_case), direction (pairs of ints) and nk wave numbers in
    [0, pi] into radius (ncases x ndirs x nk doubles) and its maximum per case
    into growth (ncases doubles); either may be None, a CUDA tensor or a host
    array."""
    cases = list(cases)
    arr = (lbm_vn_case * max(1, len(cases)))(*cases)
    flat = [int(v) for d in dirs for v in d]
    darr = (ctypes.c_int * max(1, len(flat)))(*flat)
    st = load().lbm_vn_scan(arr, len(cases), darr, len(flat) // 2, int(nk), _ptr(radius), _ptr(growth),
                            _ptr(stream))
    if st != LBM_OK:
        raise LbmError(st, load().lbm_last_error(None).decode())


def vn_case(p, state) -> lbm_vn_case:
    """lbm_vn_case of a problem description (attributes of workloads.Problem)
    linearised about the uniform state (rho, ux, uy, T)."""
    q = lbm_vn_case()
    q.b, q.tau, q.dt, q.dx = float(p.b), float(p.tau), float(p.dt), float(p.dx)
    q.dvm = lbm_dvm(p.c1, p.c2, p.eta0)
    q.diss.beta = float(p.beta)
    for i in range(9):
        q.diss.lambda_[i] = float(p.lam[i])
    for k in range(4):
        q.state[k] = float(state[k])
    return q


def vn_scan(cases, dirs=DIRECTIONS, nk: int = 31):
    """(radius, growth) as CUDA tensors, radius shaped (ncases, ndirs, nk)."""
    import torch
    cases = list(cases)
    radius = torch.empty((len(cases), len(dirs), nk), dtype=torch.float64, device="cuda")
    growth = torch.empty((len(cases),), dtype=torch.float64, device="cuda")
    lbm_vn_scan(cases, dirs, nk, radius, growth, torch.cuda.current_stream().cuda_stream)
    return radius, growth


def _bcheck(b, status):
    if status != LBM_OK:
        raise LbmError(status, load().lbm_batch_last_error(b).decode())
    return status


def lbm_batch_create(problems, prec, stream=None):
    arr = (lbm_problem * len(problems))(*problems)
    out = _VP()
    st = load().lbm_batch_create(len(problems), arr,
                                 PRECISIONS.get(prec, prec) if isinstance(prec, str) else int(prec),
                                 _ptr(stream), ctypes.byref(out))
    _bcheck(None, st)
    return out.value


def lbm_batch_destroy(b):
    load().lbm_batch_destroy(b)


def lbm_batch_last_error(b=None):
    return load().lbm_batch_last_error(b).decode()


def lbm_batch_init(b, rho, ux, uy, T):
    arrs = [(_VP * len(x))(*[_ptr(a) for a in x]) for x in (rho, ux, uy, T)]
    return _bcheck(b, load().lbm_batch_init(b, *arrs))


def lbm_batch_step(b, n):
    return _bcheck(b, load().lbm_batch_step(b, int(n)))


def lbm_batch_sync(b):
    return _bcheck(b, load().lbm_batch_sync(b))


def lbm_batch_problem(b, p):
    return load().lbm_batch_problem(b, int(p))


def lbm_batch_set_launch(b, npt, grid=0, block=0):
    l = lbm_batch_launch(int(npt), int(grid), int(block))
    return _bcheck(b, load().lbm_batch_set_launch(b, ctypes.byref(l)))


def lbm_batch_get_launch(b):
    l = lbm_batch_launch()
    _bcheck(b, load().lbm_batch_get_launch(b, ctypes.byref(l)))
    return l.as_tuple()


def lbm_batch_set_wait_limit(seconds: float) -> None:
    st = load().lbm_batch_set_wait_limit(float(seconds))
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_set_wait_limit failed")


def lbm_inject_alloc_failure(after: int) -> None:
    """The library's device allocation after the next `after` ones fails (after < 0: off)."""
    load().lbm_inject_alloc_failure(int(after))


def lbm_batch_plant_stall(b, cta: int):
    return _bcheck(b, load().lbm_batch_plant_stall(b, int(cta)))


def lbm_batch_autotune(b, steps=10):
    """Returns ((npt, grid, block) chosen, per-step ms of each candidate)."""
    best = lbm_batch_launch()
    ms = (ctypes.c_double * 8)()
    n = ctypes.c_int(0)
    _bcheck(b, load().lbm_batch_autotune(b, int(steps), ctypes.byref(best), ms, ctypes.byref(n)))
    return best.as_tuple(), list(ms[:n.value])


def lbm_batch_info(b):
    g, t, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(b, load().lbm_batch_info(b, ctypes.byref(g), ctypes.byref(t), ctypes.byref(gr)))
    return g.value, t.value, gr.value


# ------------------------------------------------------------ convenience

def make_bc(side) -> lbm_bc:
    b = lbm_bc()
    b.kind_lo = BC_KINDS[side.kind_lo]
    b.kind_hi = BC_KINDS[side.kind_hi]
    b.split0 = float(side.split0)
    b.split_speed = float(side.split_speed)
    for q in range(4):
        b.state_lo[q] = float(side.state_lo[q])
        b.state_hi[q] = float(side.state_hi[q])
    return b


def make_problem(p) -> lbm_problem:
    """lbm_problem of a problem description (attributes of workloads.Problem)."""
    q = lbm_problem()
    q.nx, q.ny = int(p.nx), int(p.ny)
    q.b, q.tau, q.dt, q.dx = float(p.b), float(p.tau), float(p.dt), float(p.dx)
    q.dvm = lbm_dvm(p.c1, p.c2, p.eta0)
    q.diss.beta = float(p.beta)
    for i in range(9):
        q.diss.lambda_[i] = float(p.lam[i])
    for k in range(4):
        q.bc[k] = make_bc(p.sides[k])
    return q


class Batch:
    """One lbm_batch for a list of problem descriptions (FP32 modes)."""

    def __init__(self, problems, precision: str = "fp32", stream=None):
        import torch
        self.problems = list(problems)
        self.precision = precision
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.handle = lbm_batch_create([make_problem(p) for p in self.problems], precision, stream)

    def close(self):
        if self.handle:
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, fields):
        """fields[p] = (rho, ux, uy, T) of problem p."""
        import torch
        ts = [[torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda") for a in fl]
              for fl in fields]
        lbm_batch_init(self.handle, *[[t[q] for t in ts] for q in range(4)])
        self._keep = ts
        return self

    def step(self, n: int):
        lbm_batch_step(self.handle, n)
        return self

    def sync(self):
        lbm_batch_sync(self.handle)

    def info(self):
        return lbm_batch_info(self.handle)

    def set_launch(self, npt: int, grid: int = 0, block: int = 0):
        lbm_batch_set_launch(self.handle, npt, grid, block)
        return self

    def get_launch(self):
        return lbm_batch_get_launch(self.handle)

    def plant_stall(self, cta: int):
        lbm_batch_plant_stall(self.handle, cta)
        return self

    def autotune(self, steps: int = 10):
        return lbm_batch_autotune(self.handle, steps)

    def moments(self, p: int):
        import torch
        prob = self.problems[p]
        ctx = lbm_batch_problem(self.handle, p)
        out = [torch.empty((prob.ny, prob.nx), dtype=torch.float32, device="cuda") for _ in range(4)]
        lbm_moments(ctx, *out)
        torch.cuda.synchronize()
        return out

    def get_f(self, p: int):
        import torch
        prob = self.problems[p]
        out = torch.empty((9, prob.ny, prob.nx), dtype=torch.float32, device="cuda")
        lbm_get_f(lbm_batch_problem(self.handle, p), out)
        torch.cuda.synchronize()
        return out


class Lattice:
    """One liblbm context for a problem (attributes of workloads.Problem).

    ``stream`` defaults to torch's current CUDA stream.  ``buffers``: optional
    pair of caller-owned CUDA tensors (or device addresses) that hold the two
    levels of f, each at least ``Lattice.level_bytes(p, precision)`` bytes
    and 256-byte aligned; the Lattice keeps them referenced while it lives
    and never frees them.  Results come back as torch CUDA tensors of the
    storage dtype."""

    @staticmethod
    def level_bytes(p, precision: str) -> int:
        return lbm_level_bytes(p.nx, p.ny, precision)

    def __init__(self, p, precision: str = "fp64", stream=None, buffers=None):
        import torch
        self.p = p
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.np_dtype = np.float64 if precision == "fp64" else np.float32
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        dvm = lbm_dvm(p.c1, p.c2, p.eta0)
        diss = lbm_dissipation()
        diss.beta = float(p.beta)
        for i in range(9):
            diss.lambda_[i] = float(p.lam[i])
        self.buffers = tuple(buffers) if buffers is not None else (None, None)
        self.ctx = lbm_create(p.nx, p.ny, p.b, p.tau, p.dt, p.dx, dvm, diss,
                              [make_bc(s) for s in p.sides], precision, stream, *self.buffers)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _dev(self, a):
        import torch
        if isinstance(a, torch.Tensor):
            return a.to(device="cuda", dtype=self.dtype).contiguous()
        return torch.as_tensor(np.ascontiguousarray(a, dtype=self.np_dtype), device="cuda")

    def init(self, rho, ux, uy, T):
        ts = [self._dev(a) for a in (rho, ux, uy, T)]
        lbm_init(self.ctx, *ts)
        self._keep = ts  # inputs live at least until the queued kernel ran
        return self

    def step(self, n: int):
        lbm_step(self.ctx, n)
        return self

    def sync(self):
        lbm_sync(self.ctx)

    def health(self) -> int:
        return lbm_health(self.ctx)

    @property
    def step_count(self) -> int:
        return lbm_step_count(self.ctx)

    def moments(self):
        import torch
        out = [torch.empty((self.p.ny, self.p.nx), dtype=self.dtype, device="cuda") for _ in range(4)]
        lbm_moments(self.ctx, *out)
        lbm_sync(self.ctx)
        return out

    def conservation(self):
        return lbm_conservation(self.ctx)

    def get_f(self):
        import torch
        out = torch.empty((9, self.p.ny, self.p.nx), dtype=self.dtype, device="cuda")
        lbm_get_f(self.ctx, out)
        torch.cuda.synchronize()
        return out

    def set_f(self, f, step: int = 0):
        t = self._dev(f)
        lbm_set_f(self.ctx, t, step)
        self._keep = [t]
        return self


__all__ = ["LbmError", "Lattice", "EXPORTS", "PRECISIONS", "load", "library_path"] + list(EXPORTS)
