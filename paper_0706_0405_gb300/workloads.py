"""Problem definitions and initial fields shaped like the paper's tests.

This module holds no arithmetic of the method (no moments, equilibrium or
stencil).  It only states grids, constants, boundary kinds and the initial
macroscopic fields (rho, ux, uy, T), with T = p / rho (R = 1), so that the
CUDA library and the oracle are driven from the same inputs.  Random draws use
numpy's PCG64 generator with a fixed seed.

Boundary sides are given in the order left (x = 0), right, bottom (y = 0),
top.  A side may switch kind and state at the along-side coordinate
``split0 + split_speed * t`` (cell-centre coordinates, x_j = (j + 1/2) dx):
below the split it uses ``kind_lo``/``state_lo``, elsewhere ``kind_hi`` /
``state_hi``.  States are (rho, ux, uy, T).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

GAMMA_AIR = 1.4
B_AIR = 2.0 / (GAMMA_AIR - 1.0)  # b = 2 / (gamma - 1), Eq. (e2) text


@dataclass(frozen=True)
class Side:
    kind_lo: str
    kind_hi: str | None = None
    split0: float = math.inf
    split_speed: float = 0.0
    state_lo: tuple = (1.0, 0.0, 0.0, 1.0)
    state_hi: tuple = (1.0, 0.0, 0.0, 1.0)

    def __post_init__(self):
        if self.kind_hi is None:
            object.__setattr__(self, "kind_hi", self.kind_lo)


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    b: float
    tau: float
    dt: float
    dx: float
    c1: float
    c2: float
    eta0: float
    beta: float
    lam: tuple
    sides: tuple
    steps: int
    setup: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def alpha(self) -> float:
        """The paper's time-step control dt = alpha dx / c2 (Sec. 3)."""
        return self.dt * self.c2 / self.dx

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def lambda_eq13(c1: float, dx: float, scale: float = 1.0) -> tuple:
    """Eq. (SEC-VON-13): lambda_0 = c1 dx, lambda_1..4 = c1 dx / 10,
    lambda_5..8 = 0, optionally times a common factor."""
    return tuple(scale * v for v in [c1 * dx] + [c1 * dx / 10.0] * 4 + [0.0] * 4)


def _ptoT(state):
    """(rho, ux, uy, p) -> (rho, ux, uy, T) with T = p / rho."""
    r, ux, uy, p = state
    return (float(r), float(ux), float(uy), float(p) / float(r))


# ---------------------------------------------------------------- Riemann tubes

def riemann(name, nx, ny, length, left, right, x_d, c1, c2, eta0, alpha=None, dt=None,
            steps=0, t_end=None, tau=None, beta=0.25, lam_scale=1.0, b=B_AIR,
            y_sides=("periodic", "periodic")) -> Problem:
    """A one-dimensional Riemann problem on an nx x ny strip of length
    ``length``; ``left``/``right`` are (rho, ux, uy, p).  Zero-gradient
    outflow in x, periodic in y unless told otherwise."""
    dx = length / nx
    if dt is None:
        dt = alpha * dx / c2
    if t_end is not None:
        steps = int(round(t_end / dt))
    sides = (Side("outflow"), Side("outflow"), Side(y_sides[0]), Side(y_sides[1]))
    return Problem(name, nx, ny, b, dt if tau is None else tau, dt, dx, c1, c2, eta0, beta,
                   lambda_eq13(c1, dx, lam_scale), sides, steps,
                   {"kind": "riemann", "left": _ptoT(left), "right": _ptoT(right), "x_d": x_d})


def sod_400x4() -> Problem:
    """Sod tube: 400 x 4, dx = 1/400, dt = tau = 1e-5, gamma = 1.4,
    (rho, u, T)_L = (1, 0, 1), (rho, u, T)_R = (0.125, 0, 0.8), diaphragm at
    x = 0.5, 2000 steps.  DVM constants c1 = 3, c2 = 9, eta0 = 5 (the set the
    paper uses for its 1000:1 tube, Fig. 10)."""
    return riemann("sod_400x4", 400, 4, 1.0, (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 0.5,
                   3.0, 9.0, 5.0, dt=1e-5, tau=1e-5, steps=2000)


def ratio1000_2000x4(alpha: float = 0.05) -> Problem:
    """Eq. (Riemann-2): (rho, u, p)_L = (1000, 0, 1000), (rho, u, p)_R =
    (1, 0, 1), dx = 0.0025 (Fig. 10), 2000 x 4 cells (length 5), diaphragm at
    2.5, c1 = 3, c2 = 9, eta0 = 5 (Fig. 10), tau = dt, t_end = 0.15."""
    return riemann("ratio1000_2000x4", 2000, 4, 5.0, (1000.0, 0.0, 0.0, 1000.0),
                   (1.0, 0.0, 0.0, 1.0), 2.5, 3.0, 9.0, 5.0, alpha=alpha, t_end=0.15)


def mach30_tube(nx: int = 1200, alpha: float = 0.05, c1: float = 33.0, c2: float = 80.0,
                eta0: float = 40.0, lam_scale: float = 2.0, steps: int = 1000) -> Problem:
    """Eq. (Riemann-1): (rho, u, p)_L = (1.4, 30, 1), (rho, u, p)_R =
    (1.4, 0, 1), dx = 0.01 (Fig. 8), diaphragm in the middle.  The paper runs
    it with c1 = 25, c2 = 50, eta0 = 30 and dt = 8e-5 (alpha = 0.4); by the
    von Neumann matrix that set grows at the inflow state (u = 30 > c1) for
    every alpha, and by 21 % per step at the right state for alpha = 0.4.
    The default here, c1 = 33, c2 = 80, eta0 = 40 with lambda = 2 x Eq. 13
    and alpha = 0.05, keeps max|omega| - 1 below 5e-6 at the left, right and
    star states.  Pass the paper's constants to run its setting."""
    return riemann(f"mach30_{nx}x4", nx, 4, nx * 0.01, (1.4, 30.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0),
                   0.5 * nx * 0.01, c1, c2, eta0, alpha=alpha, steps=steps, lam_scale=lam_scale)


def mach30_fig8(beta: float = 0.25, lam0_scale: float = 2.0, nx: int = 1600, t_end: float = 0.36,
                steps: int | None = None) -> Problem:
    """Eq. (Riemann-1) to t = 0.36 with dx = 0.01 (Figs. 8, 9): every wave
    moves right (left shock at 12, contact at 15, right shock at 18), so the
    tube is [0, 16] with the diaphragm at 6 and the fronts end near 10.3 and
    12.5.  lambda_1..8 = 2 x Eq. 13; lambda_0 = lam0_scale c1 dx (Fig. 9b
    sweeps it); beta = 0 gives the first-order upwind scheme of Fig. 9a.
    DVM constants c1 = 33, c2 = 80, eta0 = 40, alpha = 0.05, tau = dt (the
    paper's set is not stable by the von Neumann matrix, see mach30_tube)."""
    c1, dx = 33.0, 16.0 / nx
    p = riemann(f"mach30_fig8_{nx}x4", nx, 4, 16.0, (1.4, 30.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0), 6.0,
                c1, 80.0, 40.0, alpha=0.05, beta=beta, lam_scale=2.0,
                t_end=t_end if steps is None else None, steps=steps or 0)
    lam = (lam0_scale * c1 * dx,) + tuple(p.lam[1:])
    return replace(p, lam=lam)


def mach3_2048x256(steps: int = 1000) -> Problem:
    """Mach-3 tube for the adjoint: (rho, u, p)_L = (1.4, 3, 1), (rho, u, p)_R
    = (1.4, 0, 1) (sound speed 1, so Mach 3) on [0, 1] x [0, 0.125],
    dx = 1/2048, c1 = 4, c2 = 10, eta0 = 6, alpha = 0.05, tau = dt."""
    return riemann("mach3_2048x256", 2048, 256, 1.0, (1.4, 3.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0),
                   0.5, 4.0, 10.0, 6.0, alpha=0.05, steps=steps)


def batch_riemann(count: int = 256, seed: int = 0, steps: int = 1000, ny: int = 4):
    """Many Riemann tubes of uneven length, drawn from PCG64(seed):
    nx = round(exp(U[ln 256, ln 4096])) cells on [0, 1] (dx = 1 / nx), ny
    rows, diaphragm at 0.5; (rho, p)_L = (r, r) with r = exp(U[0, ln 1000]),
    (rho, p)_R = (1, 1) (T = 1 on both sides), left velocity M sqrt(1.4) with
    M ~ U[0, 30] (Mach M), right at rest.  DVM constants per tube:
    c1 = max(3, 1.1 u_L + 2, 1.05 u* + 0.5), c2 = 2.4 c1, eta0 = 1.2 c1,
    lambda = 2 x Eq. 13, dt = 0.05 dx / c2, tau = dt.  u* is the
    two-rarefaction estimate of the star velocity (Toro, Riemann Solvers and
    Numerical Methods for Fluid Dynamics, Sec. 9.4.1): the expansion of a
    dense left state can push the flow past u_L, and c1 must stay above every
    |u| the tube will see; c1 no larger than that, since a small T / c1^2
    makes the scheme less robust.  With this rule max|omega| <= 1 + 1e-5 per
    step at the left, right and star states of every tube (checked by the
    tests; the residual growth sits at the smallest wave numbers, below 1 %
    over the 1000 steps), and rho stays positive in every tube; 61 of the 256
    (dense, fast left states) pass through T < 0 behind their shocks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = np.round(np.exp(rng.uniform(math.log(256), math.log(4096), count))).astype(int)
    r = np.exp(rng.uniform(0.0, math.log(1000.0), count))
    M = rng.uniform(0.0, 30.0, count)
    out = []
    z = (GAMMA_AIR - 1.0) / (2.0 * GAMMA_AIR)
    for k in range(count):
        uL = float(M[k]) * math.sqrt(GAMMA_AIR)
        aL = aR = math.sqrt(GAMMA_AIR)           # T = 1 on both sides
        pL, pR = float(r[k]), 1.0
        p_star = ((aL + aR - 0.5 * (GAMMA_AIR - 1.0) * (0.0 - uL)) / (aL / pL ** z + aR / pR ** z)) ** (1.0 / z)
        u_star = uL - 2.0 * aL / (GAMMA_AIR - 1.0) * ((p_star / pL) ** z - 1.0)
        c1 = max(3.0, 1.1 * uL + 2.0, 1.05 * u_star + 0.5)
        out.append(riemann(f"tube{k}_{L[k]}x{ny}", int(L[k]), ny, 1.0, (float(r[k]), uL, 0.0, float(r[k])),
                           (1.0, 0.0, 0.0, 1.0), 0.5, c1, 2.4 * c1, 1.2 * c1, alpha=0.05, steps=steps,
                           lam_scale=2.0))
    return out


# ------------------------------------------------------- double Mach reflection

DMR_PRE = (1.4, 0.0, 0.0, 1.0)       # (rho, u, v, p) ahead of the shock
DMR_POST_SPEED = 8.25                # Mach-10 shock into DMR_PRE: rho 8, |u| 8.25, p 116.5
DMR_POST = (8.0, DMR_POST_SPEED * math.cos(math.pi / 6), -DMR_POST_SPEED * math.sin(math.pi / 6),
            116.5)
DMR_SHOCK_SPEED = 10.0
DMR_X0 = 1.0 / 6.0                   # where the shock meets the wall at t = 0


def dmr(ny: int = 1024, alpha: float = 0.1, lam_scale: float = 2.0, t_end: float = 0.2,
        steps: int | None = None, c1: float = 10.0, c2: float = 20.0, eta0: float = 15.0,
        x0: float = DMR_X0, dt: float | None = None) -> Problem:
    """Double Mach reflection of a Mach-10 shock (Sec. 4.2, Fig. 12), in the
    [0, 4] x [0, 1] geometry with the reflecting wall from x = 1/6 and the shock
    at 60 degrees to the wall, dx = 1/ny, dt = 0.1 dx / c2, to t = 0.2.
    DVM constants c1 = 10, c2 = 20, eta0 = 15 (the paper's Fig. 11 set) and
    lambda = 2 x Eq. (SEC-VON-13): with the Fig. 12 set (8, 16, 10) the
    post-shock speed 8.25 and the Mach-stem flow (about 12) exceed c1 and the
    temperature goes negative at the shock foot; the set used here has
    max|omega| = 1 for every state of the flow.
    Left: Dirichlet post-shock.  Right: zero-gradient outflow.  Bottom:
    Dirichlet post-shock for x < 1/6, reflecting wall beyond.  Top: the exact
    shock position x_s(t) = 1/6 + (y + 20 t) / sqrt(3) at the ghost row's
    height, post-shock state before it and pre-shock state after it.  ``x0``
    moves the wall start (and the shock's foot); ``dt`` overrides alpha."""
    nx, dx = 4 * ny, 1.0 / ny
    if dt is None:
        dt = alpha * dx / c2
    post, pre = _ptoT(DMR_POST), _ptoT(DMR_PRE)
    s3 = math.sqrt(3.0)
    y_ghost_top = (ny + 0.5) * dx
    sides = (
        Side("dirichlet", state_lo=post, state_hi=post),
        Side("outflow"),
        Side("dirichlet", "reflect", x0, 0.0, post, post),
        Side("dirichlet", "dirichlet", x0 + y_ghost_top / s3, 2.0 * DMR_SHOCK_SPEED / s3,
             post, pre),
    )
    n = int(round(t_end / dt)) if steps is None else steps
    return Problem(f"dmr_{nx}x{ny}", nx, ny, B_AIR, dt, dt, dx, c1, c2, eta0, 0.25,
                   lambda_eq13(c1, dx, lam_scale), sides, n,
                   {"kind": "dmr", "pre": pre, "post": post, "x0": x0,
                    "slope": 1.0 / s3})


def dmr_paper(alpha: float = 0.1, lam_scale: float = 2.0, t_end: float = 0.2, steps: int | None = None,
              c1: float = 10.0, c2: float = 20.0, eta0: float = 15.0, dt: float | None = None) -> Problem:
    """The paper's own double-Mach-reflection run (Sec. 4.2, Fig. 12):
    dx = dy = 0.01 on [0, 4] x [0, 1] (400 x 100 cells) with the reflecting
    wall from 20 mesh lengths (x = 0.2).  The paper's constants c1 = 8,
    c2 = 16, eta0 = 10, dt = 2e-4 can be passed; by default the vetted set of
    ``dmr`` is used, to the Woodward-Colella time t = 0.2."""
    p = dmr(100, alpha=alpha, lam_scale=lam_scale, t_end=t_end, steps=steps, c1=c1, c2=c2, eta0=eta0,
            x0=0.2, dt=dt)
    return replace(p, name="dmr_paper_400x100")


def regular_reflection(ny: int = 300, alpha: float = 0.1, lam_scale: float = 2.0,
                       t_end: float = 2.5, steps: int | None = None) -> Problem:
    """Steady regular reflection of a 30-degree shock (Sec. 4.2, Fig. 11,
    Eq. Riemann-3): domain 9 x 3 on a 3 ny x ny grid (900 x 300, dx = 0.01 by
    default), Mach-10 inflow (rho, u, v, p) = (1, 10, 0, 1/1.4) on the left
    and as the initial state everywhere, the post-shock state
    (5, 8, -2 sqrt(3), 29/1.4) (printed as (5.0, 8.0, -3.4641, 20.7143)) on
    the top, a reflecting wall at the bottom and zero-gradient outflow on the
    right; c1 = 10, c2 = 20, eta0 = 15 (Fig. 11).  The paper's dt = 1.5e-4 is
    alpha = 0.3, which grows at the inflow state by the von Neumann matrix;
    alpha = 0.1 with lambda = 2 x Eq. 13 is neutral at all three states of the
    exact solution."""
    nx, dx = 3 * ny, 3.0 / ny
    c1, c2, eta0 = 10.0, 20.0, 15.0
    dt = alpha * dx / c2
    inflow = _ptoT((1.0, 10.0, 0.0, 1.0 / 1.4))
    top = _ptoT((5.0, 8.0, -2.0 * math.sqrt(3.0), 29.0 / 1.4))
    sides = (Side("dirichlet", state_lo=inflow, state_hi=inflow), Side("outflow"), Side("reflect"),
             Side("dirichlet", state_lo=top, state_hi=top))
    n = int(round(t_end / dt)) if steps is None else steps
    return Problem(f"regref_{nx}x{ny}", nx, ny, B_AIR, dt, dt, dx, c1, c2, eta0, 0.25,
                   lambda_eq13(c1, dx, lam_scale), sides, n, {"kind": "uniform", "state": inflow})


def uniform(nx, ny, state, c1=3.0, c2=9.0, eta0=5.0, dx=0.01, alpha=0.05, tau=None,
            beta=0.25, lam_scale=1.0, sides=None, b=B_AIR, steps=100) -> Problem:
    """A uniform state (rho, ux, uy, T) (for invariance tests)."""
    dt = alpha * dx / c2
    if sides is None:
        sides = (Side("periodic"),) * 4
    return Problem(f"uniform_{nx}x{ny}", nx, ny, b, dt if tau is None else tau, dt, dx, c1, c2,
                   eta0, beta, lambda_eq13(c1, dx, lam_scale), sides, steps,
                   {"kind": "uniform", "state": tuple(float(v) for v in state)})


# -------------------------------------------------------------- initial fields

def centres(p: Problem):
    """Cell-centre coordinates (x, y), each (ny, nx)."""
    x = (np.arange(p.nx) + 0.5) * p.dx
    y = (np.arange(p.ny) + 0.5) * p.dx
    return np.meshgrid(x, y)


def initial_fields(p: Problem, seed: int | None = None, sigma: float = 0.0):
    """(rho, ux, uy, T) at t = 0, float64 arrays (ny, nx).  With ``sigma`` > 0
    each node gets an independent Gaussian perturbation of standard deviation
    sigma times the local rho, the local T and max(|u_L|, 1) for the
    velocities (PCG64, ``seed``)."""
    x, y = centres(p)
    s = p.setup
    kind = s.get("kind")
    if kind == "riemann":
        left = x < s["x_d"]
        fields = [np.where(left, s["left"][q], s["right"][q]) for q in range(4)]
    elif kind == "dmr":
        post = x < s["x0"] + s["slope"] * y
        fields = [np.where(post, s["post"][q], s["pre"][q]) for q in range(4)]
    elif kind == "uniform":
        fields = [np.full((p.ny, p.nx), s["state"][q]) for q in range(4)]
    else:
        raise ValueError(f"unknown setup {kind!r}")
    fields = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
    if sigma > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        uscale = max(abs(s.get("left", (0, 1.0))[1]), 1.0)
        scales = (fields[0], uscale, uscale, fields[3])
        fields = [f + sigma * sc * rng.standard_normal(f.shape) for f, sc in zip(fields, scales)]
    return tuple(fields)
