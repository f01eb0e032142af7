"""Pins of the oracle's adjoint (the transpose of the linearised step of
Eq. SEC-VON-11): the collision Jacobian against the independent complex-step
one, dot-product tests against central differences of the forward oracle for
every boundary kind, the tau derivative, and the gradient of a whole run
against finite differences of the loss."""
import numpy as np
import pytest

import oracle
from oracle import vonneumann as vn
from paper_0706_0405_gb300 import workloads as W
from paper_0706_0405_gb300.workloads import Side


def test_feq_jacobian_matches_complex_step():
    rng = np.random.Generator(np.random.PCG64(2))
    for _ in range(10):
        st = (rng.uniform(0.5, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.3, 2))
        p = W.uniform(2, 2, st, c1=3.0, c2=8.0, eta0=4.0)
        f = oracle.feq(p, *st) * (1 + 0.05 * rng.standard_normal(9))  # off equilibrium
        m = oracle.moments(p, f)
        Jc = oracle.feq_jacobian(p, f)
        # complex step of f -> feq(moments(f)) at f (not at an equilibrium)
        Jn = np.zeros((9, 9))
        for j in range(9):
            fp = f.astype(complex)
            fp[j] += 1e-30j
            Jn[:, j] = np.imag(vn.feq_state(*vn.moments_of(fp, p.b, p.c1, p.c2, p.eta0), p.b,
                                            p.c1, p.c2, p.eta0)) / 1e-30
        assert np.allclose(Jc, Jn, rtol=1e-11, atol=1e-12 * np.abs(Jn).max()), m


SIDES = {
    "periodic": (Side("periodic"),) * 4,
    "mixed": (Side("outflow"), Side("reflect"),
              Side("dirichlet", "reflect", 0.05, 0.0, (1.3, 0.4, -0.2, 1.1)),
              Side("dirichlet", "outflow", 0.08, 0.5, (0.9, 0.2, 0.1, 0.8))),
    "reflect": (Side("reflect"),) * 4,
}


def _state(p, rng):
    f = oracle.empty_state(p)
    base = oracle.feq(p, 1.0, 0.3, -0.2, 1.0)
    oracle.interior(f)[:] = base[:, None, None] * (1 + 0.1 * rng.standard_normal((9, p.ny, p.nx)))
    return f


def _step(p, f, n=3):
    g = f.copy()
    oracle.run(p, g, 1, n)
    return oracle.interior(g).copy()


@pytest.mark.parametrize("kind", sorted(SIDES))
def test_adjoint_step_dot_product(kind):
    """<J d, w> from central differences of the forward step equals
    <d, J^T w> from the adjoint step."""
    rng = np.random.Generator(np.random.PCG64(len(kind)))
    p = W.uniform(9, 7, (1.0, 0.0, 0.0, 1.0), dx=0.1, alpha=0.2, sides=SIDES[kind], lam_scale=2.0)
    p = p.with_(tau=p.dt / 0.8)
    f = _state(p, rng)
    d = oracle.empty_state(p) * 0.0
    oracle.interior(d)[:] = rng.standard_normal((9, p.ny, p.nx))
    w = oracle.empty_state(p) * 0.0
    oracle.interior(w)[:] = rng.standard_normal((9, p.ny, p.nx))
    eps = 1e-6
    jd = (_step(p, f + eps * d) - _step(p, f - eps * d)) / (2 * eps)
    lhs = np.sum(jd * oracle.interior(w))
    abar, _ = oracle.adjoint_step(p, f.copy(), 3, w)
    rhs = np.sum(oracle.interior(d) * oracle.interior(abar))
    assert abs(lhs - rhs) <= 1e-8 * max(abs(lhs), 1.0), (lhs, rhs)
    assert np.all(abar[:, 0, :] == 0) and np.all(abar[:, :, 0] == 0)  # ghosts carry nothing


def test_adjoint_step_tau_derivative():
    rng = np.random.Generator(np.random.PCG64(9))
    p = W.uniform(8, 5, (1.0, 0.0, 0.0, 1.0), dx=0.1, alpha=0.2, sides=SIDES["mixed"])
    tau = p.dt / 0.7
    f = _state(p, rng)
    w = oracle.empty_state(p) * 0.0
    oracle.interior(w)[:] = rng.standard_normal((9, p.ny, p.nx))
    h = tau * 1e-6
    up = _step(p.with_(tau=tau + h), f)
    dn = _step(p.with_(tau=tau - h), f)
    lhs = np.sum((up - dn) / (2 * h) * oracle.interior(w))
    _, dtau = oracle.adjoint_step(p.with_(tau=tau), f.copy(), 3, w)
    assert dtau == pytest.approx(lhs, rel=1e-7)


def _loss_run(p, fields, steps, target):
    f = oracle.init(p, *fields)
    oracle.run(p, f, steps)
    rho = oracle.fields(p, f)[0]
    return 0.5 * np.sum((rho - target) ** 2)


@pytest.mark.slow
def test_adjoint_run_matches_finite_differences():
    """dL/d(initial fields) and dL/d tau of L = 1/2 sum (rho_N - rho_target)^2
    for a perturbed Mach-3 tube, against central differences of the loss."""
    p = W.riemann("m3", 40, 4, 1.0, (1.4, 3.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0), 0.5, 4.0, 10.0,
                  6.0, alpha=0.1, steps=30)
    p = p.with_(tau=p.dt / 0.9)
    fields = W.initial_fields(p, seed=0, sigma=0.01)
    target = W.initial_fields(p, seed=1, sigma=0.01)[0]
    f = oracle.init(p, *fields)
    oracle.run(p, f, p.steps)
    rho = oracle.fields(p, f)[0]
    qbar = np.zeros((4, p.ny, p.nx))
    qbar[0] = rho - target
    grads, dtau, _ = oracle.adjoint_run(p, fields, p.steps, qbar)
    rng = np.random.Generator(np.random.PCG64(4))
    for m in range(4):
        for _ in range(3):
            k, j = rng.integers(p.ny), rng.integers(p.nx)
            h = 1e-6 * max(1.0, abs(fields[m][k, j]))
            fp = [a.copy() for a in fields]
            fm = [a.copy() for a in fields]
            fp[m][k, j] += h
            fm[m][k, j] -= h
            fd = (_loss_run(p, fp, p.steps, target) - _loss_run(p, fm, p.steps, target)) / (2 * h)
            assert grads[m, k, j] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(fd))), (m, k, j)
    h = p.tau * 1e-6
    fd = (_loss_run(p.with_(tau=p.tau + h), fields, p.steps, target)
          - _loss_run(p.with_(tau=p.tau - h), fields, p.steps, target)) / (2 * h)
    assert dtau == pytest.approx(fd, rel=1e-5)
