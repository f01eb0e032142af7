"""The batched von Neumann scanner (lbm_vn_scan) against the oracle's
amplification matrix (Sec. 3, Eqs. SEC-VON-8, 9, 12): the GPU builds G(k)
from the step's folded stencil weights and the chain-rule Jacobian of the
equilibrium and reduces it by Hessenberg-QR; the oracle builds it from the
printed symbol phi(k), a complex-step Jacobian and numpy's eigenvalues."""
import math

import numpy as np
import pytest

from oracle import gasdynamics as gd
from oracle import vonneumann as vn
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import stability
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DIRS = lbm.DIRECTIONS


def _oracle_radius(p, state, nk):
    return np.array([vn.growth_curve(state, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta,
                                     np.array(p.lam), d, nk)[1] for d in DIRS])


def _cases(seed=0, count=48):
    """Random cases spanning the paper's parameter ranges: c1 in [2, 30],
    c2 / c1 in [1.5, 3] or (0.3, 0.8), eta0 in [2, 40], alpha in [0.02, 0.8],
    beta in [0, 0.5], lambda = s x Eq. 13 with s in [0, 3], tau = dt or a
    few dt; states with |u| up to 1.2 c1 and T in [0.1, 50]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        c1 = rng.uniform(2, 30)
        c2 = c1 * (rng.uniform(1.5, 3.0) if k % 5 else rng.uniform(0.3, 0.8))
        dx = 10.0 ** rng.uniform(-3, -1)
        dt = rng.uniform(0.02, 0.8) * dx / c2
        p = W.Problem("vn", 1, 1, 2.0 / (rng.choice([1.4, 5 / 3, 1.1]) - 1.0),
                      dt * (1.0 if k % 3 else rng.uniform(1, 5)), dt, dx, c1, c2, rng.uniform(2, 40),
                      rng.uniform(0, 0.5), W.lambda_eq13(c1, dx, rng.uniform(0, 3)), (), 0)
        th = rng.uniform(0, 2 * np.pi)
        u = rng.uniform(0, 1.2) * c1
        st = (rng.uniform(0.1, 10), u * math.cos(th), u * math.sin(th), rng.uniform(0.1, 50))
        out.append((p, st))
    return out


def test_scan_matches_oracle_on_random_cases():
    cases = _cases()
    nk = 31
    radius, growth = lbm.vn_scan([lbm.vn_case(p, s) for p, s in cases], DIRS, nk)
    radius, growth = radius.cpu().numpy(), growth.cpu().numpy()
    for c, (p, s) in enumerate(cases):
        ref = _oracle_radius(p, s, nk)
        assert np.max(np.abs(radius[c] - ref) / ref) <= 1e-10, (c, np.max(np.abs(radius[c] - ref)))
        assert growth[c] == np.max(radius[c])


def test_scan_matches_oracle_on_figure_parameters(paper_values):
    rho, T, u1, u2 = paper_values["fig2_rho_T_u1_u2"]
    c1, c2, e0 = paper_values["fig2_c1_c2_eta0"]
    nk = int(paper_values["kdx_points"][0])
    cases = []
    for alpha in (0.1, 0.3, 0.45, 0.6):
        for scale in (0.0, 1.0):
            for beta in (0.0, 0.25, 0.5):
                dt = alpha * 0.01 / c2
                p = W.Problem("fig", 1, 1, 5.0, dt, dt, 0.01, c1, c2, e0, beta,
                              W.lambda_eq13(c1, 0.01, scale), (), 0)
                cases.append((p, (rho, u1, u2, T)))
    radius, _ = lbm.vn_scan([lbm.vn_case(p, s) for p, s in cases], DIRS, nk)
    radius = radius.cpu().numpy()
    for c, (p, s) in enumerate(cases):
        ref = _oracle_radius(p, s, nk)
        assert np.max(np.abs(radius[c] - ref) / ref) <= 1e-10


def test_scan_at_k_zero_is_one_for_conserved_modes():
    """k = 0 (nk = 1): G(0) = (1 - omega) I + omega J with J a projection of
    rank 4 (Eqs. e4, e5, e7 are conserved), so max|eig| = 1 exactly up to
    round-off for any omega in (0, 1]."""
    cases = [lbm.vn_case(p, s) for p, s in _cases(seed=3, count=16)]
    _, growth = lbm.vn_scan(cases, DIRS, 1)
    assert np.max(np.abs(growth.cpu().numpy() - 1.0)) <= 1e-12


def test_growth_to_host_and_device_agree():
    import torch
    cases = [lbm.vn_case(p, s) for p, s in _cases(seed=5, count=8)]
    host = np.zeros(8)
    lbm.lbm_vn_scan(cases, DIRS, 31, growth=host)
    dev = torch.empty(8, dtype=torch.float64, device="cuda")
    lbm.lbm_vn_scan(cases, DIRS, 31, growth=dev)
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())


def test_batch_tubes_are_vetted_on_the_gpu():
    """Every tube of the batched workload (all 256, not a sample) has
    max|eig G| <= 1 + 1e-5 per step at its left, right and both star states,
    and the scan agrees with the oracle's on every 16th tube."""
    cases = []
    for p in W.batch_riemann():
        L, R = p.setup["left"], p.setup["right"]
        WL, WR = (L[0], L[1], L[0] * L[3]), (R[0], R[1], R[0] * R[3])
        ps, us = gd.riemann_star(WL, WR, 1.4)
        s = gd.riemann_sample(WL, WR, 1.4, [us - 1e-9, us + 1e-9])
        for st in (L, R, (s[0, 0], us, 0.0, s[2, 0] / s[0, 0]), (s[0, 1], us, 0.0, s[2, 1] / s[0, 1])):
            cases.append(lbm.vn_case(p, st))
    g = stability.max_growth(cases)
    assert np.all(g <= 1.0 + 1e-5), np.max(g)
    probs = W.batch_riemann()
    for t in range(0, 256, 16):
        p = probs[t]
        for j in range(4):
            c = cases[4 * t + j]
            st = tuple(c.state)
            ref = vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta, np.array(p.lam))
            assert abs(g[4 * t + j] - ref) <= 1e-10 * ref


def test_largest_stable_alpha_matches_oracle():
    """The time-step choice: the largest alpha of a grid whose G does not
    grow at the tube's states, chosen from the GPU scan, equals the choice
    made with the oracle's scan."""
    alphas = np.round(np.arange(0.05, 1.01, 0.05), 2)
    for p in W.batch_riemann()[:6]:
        L, R = p.setup["left"], p.setup["right"]
        states = [L, R]
        got = stability.largest_stable_alpha(p, states, alphas, tol=1e-9)
        ok = []
        for a in alphas:
            dt = a * p.dx / p.c2
            g = max(vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, dt, p.dx, dt, p.beta, np.array(p.lam))
                    for st in states)
            if g <= 1.0 + 1e-9:
                ok.append(float(a))
        assert got == (max(ok) if ok else None), (p.name, got, ok)
