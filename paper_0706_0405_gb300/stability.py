"""Time-step selection from the von Neumann analysis of Sec. 3, on the GPU.

The paper picks dt, c1, c2, eta0 and lambda from curves of max|eig G(k)|
(Figs. 2-7); ``largest_stable_alpha`` does that choice for a problem: it
scans candidate alpha = c2 dt / dx (with tau = dt) over the states the flow
will visit and keeps the largest one whose amplification matrix does not
grow.  All eigenvalue work runs in ``lbm_vn_scan``; this module only builds
the cases and reads the answer.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import lbm


def max_growth(cases, dirs=lbm.DIRECTIONS, nk: int = 31) -> np.ndarray:
    """max|eig G| over dirs and nk wave numbers for every lbm_vn_case."""
    cases = list(cases)
    out = np.zeros(len(cases))
    if cases:
        lbm.lbm_vn_scan(cases, dirs, nk, growth=out)
    return out


def largest_stable_alpha(p, states, alphas, tol: float = 1e-9, nk: int = 31,
                         dirs=lbm.DIRECTIONS):
    """Largest alpha in ``alphas`` for which dt = alpha dx / c2, tau = dt keeps
    max|eig G| <= 1 + tol at every state (rho, ux, uy, T) in ``states``, or
    None if none does.  ``p`` (a workloads.Problem) carries the other
    constants."""
    alphas = sorted(float(a) for a in alphas)
    cases = []
    for a in alphas:
        dt = a * p.dx / p.c2
        q = replace(p, dt=dt, tau=dt)
        cases += [lbm.vn_case(q, s) for s in states]
    g = max_growth(cases, dirs, nk).reshape(len(alphas), len(states)).max(axis=1)
    ok = [a for a, v in zip(alphas, g) if v <= 1.0 + tol]
    return max(ok) if ok else None
