"""The GPU adjoint (through the C ABI) against the oracle adjoint and against
central finite differences of the GPU forward run."""
import numpy as np
import pytest

import oracle
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W
from paper_0706_0405_gb300.workloads import Side

pytestmark = pytest.mark.gpu

MIXED = (Side("outflow"), Side("reflect"),
         Side("dirichlet", "reflect", 0.05, 0.0, (1.3, 0.4, -0.2, 1.1)),
         Side("dirichlet", "outflow", 0.08, 0.5, (0.9, 0.2, 0.1, 0.8)))


def _random_state(p, rng):
    base = oracle.feq(p, 1.0, 0.3, -0.2, 1.0)
    return base[:, None, None] * (1 + 0.1 * rng.standard_normal((9, p.ny, p.nx)))


@pytest.mark.parametrize("sides", [MIXED, (Side("periodic"),) * 4, (Side("reflect"),) * 4])
def test_one_adjoint_step_matches_oracle_fp64(sides):
    rng = np.random.Generator(np.random.PCG64(11))
    p = W.uniform(13, 7, (1.0, 0.0, 0.0, 1.0), dx=0.1, alpha=0.2, sides=sides, lam_scale=2.0)
    p = p.with_(tau=p.dt / 0.8)
    f0 = _random_state(p, rng)
    w = rng.standard_normal((9, p.ny, p.nx))
    n = 3
    with lbm.Lattice(p, "fp64") as lat:
        lat.set_f(f0, n)
        lbm.lbm_record(lat.ctx, 1)
        lat.step(1)
        abar = w.copy()
        dtau = lbm.lbm_adjoint_step(lat.ctx, 1, abar)
        assert lat.step_count == n
    state = oracle.empty_state(p)
    oracle.interior(state)[:] = f0
    want, want_tau = oracle.adjoint_step(p, state, n, np.pad(w, ((0, 0), (1, 1), (1, 1))))
    wi = oracle.interior(want)
    assert np.max(np.abs(abar - wi)) <= 1e-12 * np.max(np.abs(wi))
    assert dtau == pytest.approx(want_tau, rel=1e-11)


def _mach3(nx=40, ny=4, steps=30):
    p = W.riemann("m3", nx, ny, 1.0, (1.4, 3.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0), 0.5, 4.0, 10.0,
                  6.0, alpha=0.1, steps=steps)
    return p.with_(tau=p.dt / 0.9)


@pytest.mark.parametrize("every", [1, 7, 30, 64])
def test_checkpointed_gradient_matches_oracle_fp64(every):
    """dL/d(fields) and dL/dtau through 30 steps with checkpoints every 1, 7
    (segments not dividing the run), 30 or 64 steps, against the oracle's
    adjoint run."""
    import torch
    from paper_0706_0405_gb300 import autodiff
    p = _mach3()
    fields = W.initial_fields(p, seed=0, sigma=0.01)
    target = W.initial_fields(p, seed=1, sigma=0.01)[0]
    ts = [torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True) for a in fields]
    tau = torch.tensor(p.tau, dtype=torch.float64, requires_grad=True)
    rho, ux, uy, T = autodiff.run(p, *ts, tau, p.steps, every=every)
    loss = 0.5 * torch.sum((rho - torch.tensor(target, device="cuda")) ** 2)
    loss.backward()
    qbar = np.zeros((4, p.ny, p.nx))
    qbar[0] = rho.detach().cpu().numpy() - target
    grads, dtau, _ = oracle.adjoint_run(p, fields, p.steps, qbar)
    for m in range(4):
        g = ts[m].grad.cpu().numpy()
        assert np.max(np.abs(g - grads[m])) <= 1e-10 * max(np.max(np.abs(grads[m])), 1e-300), m
    assert float(tau.grad) == pytest.approx(dtau, rel=1e-10)


def test_adjoint_of_all_moment_outputs_matches_oracle_fp64():
    import torch
    from paper_0706_0405_gb300 import autodiff
    p = _mach3(24, 3, 12).with_(sides=MIXED)
    fields = W.initial_fields(p, seed=2, sigma=0.02)
    rng = np.random.Generator(np.random.PCG64(5))
    wq = rng.standard_normal((4, p.ny, p.nx))
    ts = [torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True) for a in fields]
    outs = autodiff.run(p, *ts, p.tau, p.steps, every=5)
    loss = sum(torch.sum(o * torch.tensor(w, device="cuda")) for o, w in zip(outs, wq))
    loss.backward()
    grads, _, _ = oracle.adjoint_run(p, fields, p.steps, wq)
    for m in range(4):
        g = ts[m].grad.cpu().numpy()
        assert np.max(np.abs(g - grads[m])) <= 1e-10 * np.max(np.abs(grads[m])), m


def _loss(p, fields, target, prec="fp64"):
    with lbm.Lattice(p, prec) as lat:
        lat.init(*fields).step(p.steps)
        rho = lat.moments()[0].double().cpu().numpy()
    return 0.5 * np.sum((rho - target) ** 2)


def _fp32_bound(g64, g32, g_delta, m):
    """The FP32 gradient's error bound for field m.  The FP32 gradient is
    Jhat^T (rho32 - target) against J^T (rho64 - target) in FP64, so
      g32 - g64 = J^T (rho32 - rho64) + (Jhat - J)^T (rho32 - target):
    the FP32 forward error of the final density pushed back through the exact
    adjoint (g_delta, computed in FP64 with that error as the seed), plus the
    FP32 adjoint's own error.  That is its roundings, about three FP32 ulps
    (6e-8 each) of the adjoint state per step, 2e-4 of |g| if all 1000 steps
    of the full-size run added up coherently, and its linearisation about the
    FP32 states (state error ~1e-5).  Bound: |g_delta| + 2e-4 |g|.  Measured
    on the full-size run: own error at most 2.2e-5 of |g|; total error
    1e-4 (plain FP32) and 2e-5 (double-float T)."""
    err = np.linalg.norm(g32[m] - g64[m])
    bound = np.linalg.norm(g_delta[m]) + 2e-4 * np.linalg.norm(g64[m])
    return err, bound


def test_mach3_2048x256_gradient_against_finite_differences():
    """The adjoint configuration at full size: Mach-3 tube 2048 x 256, 1000
    steps, checkpoint every 50, loss = 1/2 sum (rho_final - rho_target)^2 with
    target and start from independently perturbed states (sigma 1 %).  The
    FP64 adjoint's directional derivatives (random directions in each initial
    field, and tau) agree with central differences of the FP64 forward run to
    1e-4 relative.  The FP32 adjoints (plain FP32 and the double-float
    temperature mode) agree with the FP64 one within the bound of
    _fp32_bound."""
    import torch
    from paper_0706_0405_gb300 import autodiff
    p = W.mach3_2048x256()
    fields = W.initial_fields(p, seed=0, sigma=0.01)
    target = W.initial_fields(p, seed=1, sigma=0.01)[0]
    tgt = torch.tensor(target, device="cuda")
    grads, rho_final = {}, {}
    for prec in ("fp64", "fp32", "fp32_tdf"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        ts = [torch.tensor(a, dtype=dt, device="cuda", requires_grad=True) for a in fields]
        tau = torch.tensor(p.tau, dtype=torch.float64, requires_grad=True)
        rho, _, _, _ = autodiff.run(p, *ts, tau, p.steps, every=50, precision=prec)
        loss = 0.5 * torch.sum((rho.double() - tgt) ** 2)
        loss.backward()
        grads[prec] = ([t.grad.double().cpu().numpy() for t in ts], float(tau.grad))
        rho_final[prec] = rho.detach().double()
    g64, dtau64 = grads["fp64"]
    rng = np.random.Generator(np.random.PCG64(8))
    for m in range(4):
        d = rng.standard_normal((p.ny, p.nx))
        h = 1e-6 * max(1.0, np.max(np.abs(fields[m])))
        fp = [a.copy() for a in fields]
        fm = [a.copy() for a in fields]
        fp[m] = fp[m] + h * d
        fm[m] = fm[m] - h * d
        fd = (_loss(p, fp, target) - _loss(p, fm, target)) / (2 * h)
        ad = float(np.sum(g64[m] * d))
        assert ad == pytest.approx(fd, rel=1e-4), m
    h = p.tau * 1e-6
    fd = (_loss(p.with_(tau=p.tau + h), fields, target)
          - _loss(p.with_(tau=p.tau - h), fields, target)) / (2 * h)
    assert dtau64 == pytest.approx(fd, rel=1e-4)
    for prec in ("fp32", "fp32_tdf"):
        # J^T (rho32 - rho64) in FP64: the gradient of sum(delta * rho_final)
        delta = rho_final[prec] - rho_final["fp64"]
        ts = [torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True) for a in fields]
        rho, _, _, _ = autodiff.run(p, *ts, p.tau, p.steps, every=50)
        torch.sum(rho * delta).backward()
        g_delta = [t.grad.cpu().numpy() for t in ts]
        g32, _ = grads[prec]
        for m in range(4):
            err, bound = _fp32_bound(g64, g32, g_delta, m)
            assert err <= bound, (prec, m, err / np.linalg.norm(g64[m]), bound / np.linalg.norm(g64[m]))


@pytest.mark.parametrize("prec", ["fp32", "fp32_tdf", "fp32_cons"])
def test_fp32_gradient_of_a_reduced_mach3_tube_against_the_oracle_adjoint(prec):
    """The FP32 GPU gradient (checkpointed, tile kernels) of a reduced Mach-3
    tube (256 x 8, 200 steps) against the FP64 oracle's adjoint run, within
    the bound of _fp32_bound, with the forward error's share taken from the
    oracle's adjoint seeded with it."""
    import torch
    from paper_0706_0405_gb300 import autodiff
    p = _mach3(256, 8, 200)
    fields = W.initial_fields(p, seed=0, sigma=0.01)
    target = W.initial_fields(p, seed=1, sigma=0.01)[0]
    ts = [torch.tensor(a, dtype=torch.float32, device="cuda", requires_grad=True) for a in fields]
    rho, _, _, _ = autodiff.run(p, *ts, p.tau, p.steps, every=16, precision=prec)
    loss = 0.5 * torch.sum((rho.double() - torch.tensor(target, device="cuda")) ** 2)
    loss.backward()
    g32 = [t.grad.double().cpu().numpy() for t in ts]
    f = oracle.init(p, *fields)
    assert oracle.run(p, f, p.steps) == 0
    rho64 = oracle.fields(p, f)[0]
    qbar = np.zeros((4, p.ny, p.nx))
    qbar[0] = rho64 - target
    g64, _, _ = oracle.adjoint_run(p, fields, p.steps, qbar)
    qbar[0] = rho.detach().double().cpu().numpy() - rho64
    g_delta, _, _ = oracle.adjoint_run(p, fields, p.steps, qbar)
    for m in range(4):
        err, bound = _fp32_bound(g64, g32, g_delta, m)
        assert err <= bound, (m, err / np.linalg.norm(g64[m]), bound / np.linalg.norm(g64[m]))


def test_adjoint_needs_a_recording():
    p = _mach3()
    with lbm.Lattice(p, "fp64") as lat:
        lat.init(*W.initial_fields(p)).step(3)
        abar = np.zeros((9, p.ny, p.nx))
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_adjoint_step(lat.ctx, 1, abar)
        assert ei.value.status == lbm.LBM_E_STATE
        lbm.lbm_record(lat.ctx, 2)
        lat.step(3)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_adjoint_step(lat.ctx, 4, abar)
        assert ei.value.status == lbm.LBM_E_INVAL
        lbm.lbm_adjoint_step(lat.ctx, 3, abar)  # host array, exactly what was recorded
        assert lat.step_count == 3


@pytest.mark.parametrize("sides", [MIXED, (Side("periodic"),) * 4, (Side("reflect"),) * 4])
def test_fp32_tile_adjoint_matches_oracle_and_simple_kernel(sides):
    """One FP32 adjoint step on a 150 x 37 grid (tiles of 64 x 4 with ragged
    edges, several CTAs) through the tile kernel (the default launch) and
    through the thread-per-node kernel (launch variant 0): both equal the
    FP64 oracle adjoint to FP32 accuracy, and each other to a few ulp."""
    rng = np.random.Generator(np.random.PCG64(12))
    p = W.uniform(150, 37, (1.0, 0.0, 0.0, 1.0), dx=0.1, alpha=0.2, sides=sides, lam_scale=2.0)
    p = p.with_(tau=p.dt / 0.8)
    f0 = _random_state(p, rng)
    w = rng.standard_normal((9, p.ny, p.nx))
    n = 5
    out = {}
    for variant in (3, 0):
        with lbm.Lattice(p, "fp32_cons") as lat:
            lbm.lbm_set_launch(lat.ctx, variant)
            lat.set_f(f0.astype(np.float32), n)
            lbm.lbm_record(lat.ctx, 1)
            lat.step(1)
            abar = w.astype(np.float32)
            dtau = lbm.lbm_adjoint_step(lat.ctx, 1, abar)
            out[variant] = (abar.astype(np.float64), dtau)
    state = oracle.empty_state(p)
    oracle.interior(state)[:] = f0.astype(np.float32).astype(np.float64)
    want, want_tau = oracle.adjoint_step(p, state, n, np.pad(w.astype(np.float32).astype(np.float64),
                                                              ((0, 0), (1, 1), (1, 1))))
    wi = oracle.interior(want)
    scale = np.max(np.abs(wi))
    for variant, (abar, dtau) in out.items():
        assert np.max(np.abs(abar - wi)) <= 2e-5 * scale, variant
        assert dtau == pytest.approx(want_tau, rel=1e-4), variant
    assert np.max(np.abs(out[3][0] - out[0][0])) <= 1e-6 * scale


def _fields_from_states(p, states, z, sigma, xp):
    """Initial fields of the Mach-3 tube as functions of its left and right
    states (rho, u, T)_L, (rho, u, T)_R with the seeded perturbation z:
    rho (1 + sigma z), u + sigma max(|u_L|, 1) z, T (1 + sigma z)."""
    rL, uL, TL, rR, uR, TR = states
    x, _ = W.centres(p)
    left = x < p.setup["x_d"]
    if xp.__name__ == "torch":
        left = xp.as_tensor(left, device="cuda")
    where = (lambda c, a, b: xp.where(c, a, b))
    uscale = xp.clamp(xp.abs(uL), min=1.0) if xp.__name__ == "torch" else max(abs(uL), 1.0)
    rho = where(left, rL, rR) * (1 + sigma * z[0])
    ux = where(left, uL, uR) + sigma * uscale * z[1]
    uy = 0.0 * rho + sigma * uscale * z[2]
    T = where(left, TL, TR) * (1 + sigma * z[3])
    return rho, ux, uy, T


def test_mach3_gradient_wrt_left_and_right_states_against_finite_differences():
    """The adjoint configuration (Mach-3 tube 2048 x 256, 1000 steps,
    checkpoint every 50, 1 % seeded perturbation): dL/d(rho, u, T) of the
    left and right Riemann states through the GPU adjoint and autograd equal
    central differences of the FP64 forward run to 1e-4 relative."""
    import torch
    from paper_0706_0405_gb300 import autodiff
    p = W.mach3_2048x256()
    rng = np.random.Generator(np.random.PCG64(21))
    z = [rng.standard_normal((p.ny, p.nx)) for _ in range(4)]
    target = W.initial_fields(p, seed=1, sigma=0.01)[0]
    L, R = p.setup["left"], p.setup["right"]
    s0 = [L[0], L[1], L[3], R[0], R[1], R[3]]
    st = [torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True) for v in s0]
    zt = [torch.tensor(a, device="cuda") for a in z]
    fields = _fields_from_states(p, st, zt, 0.01, torch)
    rho, _, _, _ = autodiff.run(p, *[f.contiguous() for f in fields], p.tau, p.steps, every=50)
    loss = 0.5 * torch.sum((rho - torch.tensor(target, device="cuda")) ** 2)
    loss.backward()
    for k in range(6):
        h = 1e-6 * max(1.0, abs(s0[k]))
        sp, sm = list(s0), list(s0)
        sp[k] += h
        sm[k] -= h
        fp = [np.ascontiguousarray(a) for a in _fields_from_states(p, sp, z, 0.01, np)]
        fm = [np.ascontiguousarray(a) for a in _fields_from_states(p, sm, z, 0.01, np)]
        fd = (_loss(p, fp, target) - _loss(p, fm, target)) / (2 * h)
        assert st[k].grad.item() == pytest.approx(fd, rel=1e-4, abs=1e-8 * abs(loss.item())), k


TINY = [
    (1, 1, (Side("periodic"),) * 4),
    (1, 9, (Side("periodic"), Side("periodic"), Side("outflow"), Side("reflect"))),
    (9, 1, (Side("outflow"), Side("reflect"), Side("periodic"), Side("periodic"))),
    (70, 3, MIXED),
    (3, 70, (Side("reflect"),) * 4),
]


@pytest.mark.parametrize("nx,ny,sides", TINY)
def test_adjoint_on_one_node_one_row_and_one_column_grids(nx, ny, sides):
    """One adjoint step on grids of one node, one column, one row and thinner
    than a tile: FP64 against the oracle adjoint to 1e-12, and the FP32 tile
    and thread-per-node adjoint kernels against it to FP32 accuracy."""
    rng = np.random.Generator(np.random.PCG64(nx * 100 + ny))
    p = W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), dx=0.1, alpha=0.2, sides=sides, lam_scale=2.0)
    p = p.with_(tau=p.dt / 0.8)
    f0 = _random_state(p, rng)
    w = rng.standard_normal((9, p.ny, p.nx))
    n = 3
    state = oracle.empty_state(p)
    oracle.interior(state)[:] = f0
    want, want_tau = oracle.adjoint_step(p, state, n, np.pad(w, ((0, 0), (1, 1), (1, 1))))
    wi = oracle.interior(want)
    scale = np.max(np.abs(wi))
    with lbm.Lattice(p, "fp64") as lat:
        lat.set_f(f0, n)
        lbm.lbm_record(lat.ctx, 1)
        lat.step(1)
        abar = w.copy()
        dtau = lbm.lbm_adjoint_step(lat.ctx, 1, abar)
    assert np.max(np.abs(abar - wi)) <= 1e-12 * scale
    assert dtau == pytest.approx(want_tau, rel=1e-10, abs=1e-12 * abs(want_tau) + 1e-14)
    # FP32 against the oracle run on the FP32-rounded inputs
    state32 = oracle.empty_state(p)
    oracle.interior(state32)[:] = f0.astype(np.float32).astype(np.float64)
    want32, _ = oracle.adjoint_step(p, state32, n, np.pad(w.astype(np.float32).astype(np.float64),
                                                          ((0, 0), (1, 1), (1, 1))))
    wi32 = oracle.interior(want32)
    for variant in (3, 0):
        with lbm.Lattice(p, "fp32_cons") as lat:
            lbm.lbm_set_launch(lat.ctx, variant)
            lat.set_f(f0.astype(np.float32), n)
            lbm.lbm_record(lat.ctx, 1)
            lat.step(1)
            abar = w.astype(np.float32)
            lbm.lbm_adjoint_step(lat.ctx, 1, abar)
        assert np.max(np.abs(abar.astype(np.float64) - wi32)) <= 2e-5 * scale, variant
