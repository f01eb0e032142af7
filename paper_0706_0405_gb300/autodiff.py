"""torch.autograd binding of the hand-written adjoint (C ABI: lbm_record,
lbm_adjoint_seed, lbm_adjoint_step, lbm_feq_vjp).

``run(problem, rho0, ux0, uy0, T0, tau, steps)`` advances f^0 = f^eq(fields)
by ``steps`` steps of Eq. (SEC-VON-11) on the GPU and returns the final
(rho, ux, uy, T).  Its backward pass runs the adjoint kernels with a
checkpoint every ``every`` steps (the levels in between are recomputed), and
returns gradients for the four initial fields and for tau.  The arithmetic
happens in liblbm; this module only moves tensors and pointers.
"""
from __future__ import annotations

import torch

from . import lbm


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, ux0, uy0, T0, tau, problem, steps, every, precision):
        p = problem.with_(tau=float(tau))
        lat = lbm.Lattice(p, precision)
        fields = [lat._dev(a) for a in (rho0, ux0, uy0, T0)]
        lat.init(*fields)
        lbm.lbm_record(lat.ctx, every)
        lat.step(steps)
        out = lat.moments()
        ctx.lat = lat
        ctx.steps = steps
        ctx.fields = fields
        ctx.in_dtype = rho0.dtype
        ctx.tau_dtype = tau.dtype if torch.is_tensor(tau) else torch.float64
        return tuple(o.to(rho0.dtype) for o in out)

    @staticmethod
    def backward(ctx, g_rho, g_ux, g_uy, g_T):
        lat = ctx.lat
        p = lat.p
        dev = lambda g: None if g is None else g.to(device="cuda", dtype=lat.dtype).contiguous()
        abar = torch.empty((9, p.ny, p.nx), dtype=lat.dtype, device="cuda")
        gs = [dev(g) for g in (g_rho, g_ux, g_uy, g_T)]
        lbm.lbm_adjoint_seed(lat.ctx, *gs, abar)
        dtau = lbm.lbm_adjoint_step(lat.ctx, ctx.steps, abar)
        grads = [torch.empty_like(ctx.fields[0]) for _ in range(4)]
        lbm.lbm_feq_vjp(lat.ctx, *ctx.fields, abar, *grads)
        torch.cuda.synchronize()
        lat.close()
        ctx.lat = None
        out = [g.to(ctx.in_dtype) for g in grads]
        return (*out, torch.tensor(dtau, dtype=ctx.tau_dtype), None, None, None, None)


def run(problem, rho0, ux0, uy0, T0, tau, steps: int, every: int = 50, precision: str = "fp64"):
    """Differentiable GPU run; see the module docstring."""
    if not torch.is_tensor(tau):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    return _Run.apply(rho0, ux0, uy0, T0, tau, problem, int(steps), int(every), precision)
