"""Oracle for the KT D2V9 finite-difference lattice Boltzmann step with the
added dissipation term (Pan, Xu, Zhang & Jiang, IJMPC 2007).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is a plain,
slow, serial FP64 restatement of the paper and shares no code with the CUDA
library in ``paper_0706_0405_gb300``; neither imports the other.

Contents
--------
``kt_oracle.c`` (loaded here through ctypes)
    velocity table (Eq. e14), moments (Eqs. e4, e5, e7), equilibrium
    (Eqs. e16-e18), ghost layer from the boundary kinds, beta-upwind
    derivative (Eqs. SEC-VON-2a/2b), central second difference and the
    forward-Euler update with BGK relaxation and dissipation (Eq. SEC-VON-11).
``vonneumann.py``
    the amplification matrix G(k) of Eqs. (SEC-VON-8, 9, 12) and its spectral
    radius.
``gasdynamics.py``
    the exact Riemann solution of the Euler equations (Eq. e2) and
    Rankine-Hugoniot jump relations, used to check the oracle's runs.

Problems are passed as any object with the attributes ``nx, ny, b, tau, dt,
dx, c1, c2, eta0, beta, lam`` (9 values) and ``sides`` (4 objects with
``kind_lo, kind_hi, split0, split_speed, state_lo, state_hi``; kinds are the
strings ``periodic``, ``outflow``, ``dirichlet``, ``reflect``; order left,
right, bottom, top).
"""
from __future__ import annotations

import ctypes

import numpy as np

from .build import build_oracle

KINDS = {"periodic": 0, "outflow": 1, "dirichlet": 2, "reflect": 3}


class _Side(ctypes.Structure):
    _fields_ = [
        ("kind_lo", ctypes.c_int),
        ("kind_hi", ctypes.c_int),
        ("split0", ctypes.c_double),
        ("split_speed", ctypes.c_double),
        ("state_lo", ctypes.c_double * 4),
        ("state_hi", ctypes.c_double * 4),
    ]


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("b", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("c1", ctypes.c_double),
        ("c2", ctypes.c_double),
        ("eta0", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("lam", ctypes.c_double * 9),
        ("side", _Side * 4),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        cfgp = ctypes.POINTER(_Config)
        lib.kt_velocities.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
        lib.kt_feq.argtypes = [cfgp] + [ctypes.c_double] * 4 + [_D]
        lib.kt_moments.argtypes = [cfgp, _D, _D]
        lib.kt_field_len.argtypes = [cfgp]
        lib.kt_field_len.restype = ctypes.c_size_t
        lib.kt_fill_ghosts.argtypes = [cfgp, _D, ctypes.c_double]
        lib.kt_init.argtypes = [cfgp, _D, _D, _D, _D, _D]
        lib.kt_run.argtypes = [cfgp, _D, _D, ctypes.c_long, ctypes.c_long]
        lib.kt_run.restype = ctypes.c_long
        lib.kt_run_f32_storage.argtypes = [cfgp, _D, _D, ctypes.c_long, ctypes.c_long]
        lib.kt_run_f32_storage.restype = ctypes.c_long
        lib.kt_step_nodes.argtypes = [cfgp, _D, ctypes.c_long, _L, ctypes.c_long, _D]
        lib.kt_fields.argtypes = [cfgp, _D, _D, _D, _D, _D]
        lib.kt_sums.argtypes = [cfgp, _D, _D]
        lib.kt_feq_jacobian.argtypes = [cfgp, _D, _D]
        lib.kt_feq_vjp.argtypes = [cfgp, _D, _D, _D]
        lib.kt_moments_vjp.argtypes = [cfgp, _D, _D, _D]
        lib.kt_adjoint_step.argtypes = [cfgp, _D, ctypes.c_long, _D, _D, _D]
        lib.kt_set_threads.argtypes = [ctypes.c_int]
        lib.kt_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def config(p) -> _Config:
    """Pack a problem description (see module docstring) into the C struct."""
    c = _Config()
    c.nx, c.ny = int(p.nx), int(p.ny)
    c.b, c.tau, c.dt, c.dx = float(p.b), float(p.tau), float(p.dt), float(p.dx)
    c.c1, c.c2, c.eta0, c.beta = float(p.c1), float(p.c2), float(p.eta0), float(p.beta)
    for i in range(9):
        c.lam[i] = float(p.lam[i])
    for s in range(4):
        sd = p.sides[s]
        c.side[s].kind_lo = KINDS[sd.kind_lo]
        c.side[s].kind_hi = KINDS[sd.kind_hi]
        c.side[s].split0 = float(sd.split0)
        c.side[s].split_speed = float(sd.split_speed)
        for q in range(4):
            c.side[s].state_lo[q] = float(sd.state_lo[q])
            c.side[s].state_hi[q] = float(sd.state_hi[q])
    return c


def set_threads(n: int) -> None:
    """Threads for the row loop of ``run`` (results do not depend on it)."""
    _load().kt_set_threads(int(n))


def max_threads() -> int:
    return int(_load().kt_max_threads())


def velocities(c1: float, c2: float):
    """Eq. (e14): the nine velocities as two arrays (vx, vy)."""
    vx, vy = np.zeros(9), np.zeros(9)
    _load().kt_velocities(c1, c2, _ptr(vx), _ptr(vy))
    return vx, vy


def feq(p, rho, ux, uy, T) -> np.ndarray:
    """Eqs. (e16)-(e18) at one state."""
    out = np.zeros(9)
    c = config(p)
    _load().kt_feq(ctypes.byref(c), rho, ux, uy, T, _ptr(out))
    return out


def moments(p, f9) -> np.ndarray:
    """Eqs. (e4), (e5), (e7): (rho, ux, uy, T) of nine populations."""
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    out = np.zeros(4)
    c = config(p)
    _load().kt_moments(ctypes.byref(c), _ptr(f9), _ptr(out))
    return out


def empty_state(p) -> np.ndarray:
    return np.full((9, p.ny + 2, p.nx + 2), np.nan)


def init(p, rho, ux, uy, T) -> np.ndarray:
    """f = f^eq of the (ny, nx) fields; returns the (9, ny+2, nx+2) state with
    a NaN ghost layer."""
    c = config(p)
    f = empty_state(p)
    arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(p.ny, p.nx) for a in (rho, ux, uy, T)]
    _load().kt_init(ctypes.byref(c), *[_ptr(a) for a in arrs], _ptr(f))
    return f


def fill_ghosts(p, f: np.ndarray, t: float) -> None:
    c = config(p)
    _load().kt_fill_ghosts(ctypes.byref(c), _ptr(f), float(t))


def run(p, f: np.ndarray, nsteps: int, n0: int = 0, f32_storage: bool = False) -> int:
    """Advance f in place by nsteps steps from step index n0; returns the
    number of nodes left with rho <= 0, T <= 0 or a non-finite velocity.
    f32_storage: keep the state rounded to FP32 between steps (FP64
    arithmetic), the error floor of any FP32-storage implementation; this
    rounds f itself first."""
    c = config(p)
    work = np.empty_like(f)
    fn = _load().kt_run_f32_storage if f32_storage else _load().kt_run
    return int(fn(ctypes.byref(c), _ptr(f), _ptr(work), int(nsteps), int(n0)))


def step_nodes(p, f: np.ndarray, n: int, nodes) -> np.ndarray:
    """One step from the level-n state f (step index n) evaluated only at the
    interior nodes ``nodes`` (flat index ky * nx + kx); returns (count, 9).
    f's ghost layer is refilled in place."""
    c = config(p)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((len(nodes), 9))
    _load().kt_step_nodes(ctypes.byref(c), _ptr(f), int(n), nodes.ctypes.data_as(_L),
                          len(nodes), _ptr(out))
    return out


def fields(p, f: np.ndarray):
    """(rho, ux, uy, T), each (ny, nx)."""
    c = config(p)
    outs = [np.zeros((p.ny, p.nx)) for _ in range(4)]
    _load().kt_fields(ctypes.byref(c), _ptr(f), *[_ptr(a) for a in outs])
    return tuple(outs)


def sums(p, f: np.ndarray) -> np.ndarray:
    """Interior totals of rho, rho ux, rho uy and rho (b T + u^2)."""
    c = config(p)
    out = np.zeros(4)
    _load().kt_sums(ctypes.byref(c), _ptr(f), _ptr(out))
    return out


def feq_jacobian(p, f9) -> np.ndarray:
    """J[i, j] = d f^eq_i / d f_j at the nine populations f9 (chain rule
    through the moments)."""
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    J = np.zeros(81)
    c = config(p)
    _load().kt_feq_jacobian(ctypes.byref(c), _ptr(f9), _ptr(J))
    return J.reshape(9, 9)


def feq_vjp(p, q, abar9) -> np.ndarray:
    """sum_i abar_i d f^eq_i / d q for q = (rho, ux, uy, T)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    abar9 = np.ascontiguousarray(abar9, dtype=np.float64)
    out = np.zeros(4)
    c = config(p)
    _load().kt_feq_vjp(ctypes.byref(c), _ptr(q), _ptr(abar9), _ptr(out))
    return out


def moments_vjp(p, f9, qbar) -> np.ndarray:
    """sum_m qbar_m d q_m / d f at the populations f9."""
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    qbar = np.ascontiguousarray(qbar, dtype=np.float64)
    out = np.zeros(9)
    c = config(p)
    _load().kt_moments_vjp(ctypes.byref(c), _ptr(f9), _ptr(qbar), _ptr(out))
    return out


def adjoint_step(p, f: np.ndarray, n: int, abar_next: np.ndarray):
    """Adjoint of the step from level n (state f) to level n + 1: returns
    (abar_n, dL/dtau contribution).  f's ghost layer is refilled."""
    c = config(p)
    abar = np.zeros_like(f)
    an = np.ascontiguousarray(abar_next, dtype=np.float64)
    dtau = np.zeros(1)
    _load().kt_adjoint_step(ctypes.byref(c), _ptr(f), int(n), _ptr(an), _ptr(abar), _ptr(dtau))
    return abar, float(dtau[0])


def adjoint_run(p, initial, steps: int, qbar_final):
    """Gradient of L through `steps` steps from f^0 = f^eq(initial), given
    qbar_final = dL/d(rho, ux, uy, T) of the final level ((4, ny, nx)).
    Stores every level (small problems only).  Returns
    (dL/d fields (4, ny, nx), dL/d tau, final fields)."""
    f = init(p, *initial)
    levels = [f.copy()]
    for n in range(steps):
        g = levels[-1].copy()
        run(p, g, 1, n)
        levels.append(g)
    fin = levels[-1]
    abar = empty_state(p) * 0.0
    qb = np.asarray(qbar_final, dtype=np.float64)
    for k in range(p.ny):
        for j in range(p.nx):
            abar[:, k + 1, j + 1] = moments_vjp(p, fin[:, k + 1, j + 1], qb[:, k, j])
    dtau = 0.0
    for n in range(steps - 1, -1, -1):
        abar, dt_n = adjoint_step(p, levels[n].copy(), n, abar)
        dtau += dt_n
    grads = np.zeros((4, p.ny, p.nx))
    flds = [np.asarray(a, dtype=np.float64).reshape(p.ny, p.nx) for a in initial]
    for k in range(p.ny):
        for j in range(p.nx):
            q = [flds[m][k, j] for m in range(4)]
            grads[:, k, j] = feq_vjp(p, q, abar[:, k + 1, j + 1])
    return grads, dtau, fields(p, fin)


def interior(f: np.ndarray) -> np.ndarray:
    """The (9, ny, nx) interior of a state with ghost layer."""
    return f[:, 1:-1, 1:-1]


def default_lambda(c1: float, dx: float, scale: float = 1.0) -> np.ndarray:
    """Eq. (SEC-VON-13): lambda_0 = c1 dx, lambda_1..4 = c1 dx / 10,
    lambda_5..8 = 0 (times an optional common factor)."""
    lam = np.zeros(9)
    lam[0] = c1 * dx
    lam[1:5] = c1 * dx / 10.0
    return lam * scale


__all__ = [
    "config", "set_threads", "max_threads", "velocities", "feq", "moments", "empty_state",
    "init", "fill_ghosts", "run", "step_nodes", "fields", "sums", "interior", "default_lambda",
    "feq_jacobian", "feq_vjp", "moments_vjp", "adjoint_step", "adjoint_run",
]
