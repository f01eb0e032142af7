"""Pins of the oracle's von Neumann tool (Sec. 3, Eqs. SEC-VON-8, 9, 12) and
the qualitative claims the paper makes from it (Figs. 2-7).  The curves
themselves are not printed, so their exact values are unpinned; the
orderings stated in the text are."""
import numpy as np
import pytest

from oracle import vonneumann as vn
from paper_0706_0405_gb300 import workloads as W

B = 5.0  # gamma = 1.4


def _fig_state(paper_values):
    rho, T, u1, u2 = paper_values["fig2_rho_T_u1_u2"]
    return (rho, u1, u2, T)


def _curve(paper_values, alpha, diss=True, beta=0.25, c2=None, eta0=None, state=None, dx=0.01):
    c1, c2d, e0d = paper_values["fig2_c1_c2_eta0"]
    c2 = c2d if c2 is None else c2
    eta0 = e0d if eta0 is None else eta0
    dt = alpha * dx / c2
    lam = np.array(W.lambda_eq13(c1, dx)) if diss else np.zeros(9)
    st = _fig_state(paper_values) if state is None else state
    th, g = vn.growth_curve(st, B, c1, c2, eta0, dt, dx, dt, beta, lam,
                            npts=int(paper_values["kdx_points"][0]))
    return g


def test_eq13_defaults(paper_values):
    lam = np.array(W.lambda_eq13(10.0, 0.01)) / (10.0 * 0.01)
    assert np.allclose(lam, paper_values["eq13_lambda_over_c1dx"])


def test_jacobian_is_projection_onto_conserved_moments():
    """f -> f^eq(moments f) is idempotent with rank 4 (rho, rho u, E), so at
    k = 0 the eigenvalues of G are 1 (four times) and 1 - dt/tau (five times)."""
    st = (1.3, 0.7, -0.4, 0.9)
    J = vn.feq_jacobian(st, B, 3.0, 9.0, 5.0)
    assert np.allclose(J @ J, J, atol=1e-12)
    assert np.linalg.matrix_rank(J, tol=1e-9) == 4
    w = 0.6
    G = vn.amplification_matrix(0.0, 0.0, st, B, 3.0, 9.0, 5.0, 1e-4, 0.01, 1e-4 / w, 0.25,
                                np.array(W.lambda_eq13(3.0, 0.01)))
    ev = np.sort(np.abs(np.linalg.eigvals(G)))
    assert np.allclose(ev, sorted([1 - w] * 5 + [1.0] * 4), atol=1e-12)


def test_jacobian_matches_finite_difference_of_oracle():
    """The complex-step Jacobian agrees with central differences of the C
    oracle's f -> f^eq(moments f)."""
    import oracle
    st = (0.8, 1.1, 0.3, 1.7)
    p = W.uniform(2, 2, st)
    J = vn.feq_jacobian(st, p.b, p.c1, p.c2, p.eta0)
    f0 = oracle.feq(p, *st)
    h = 1e-6
    for j in range(9):
        fp, fm = f0.copy(), f0.copy()
        fp[j] += h
        fm[j] -= h
        col = (oracle.feq(p, *oracle.moments(p, fp)) - oracle.feq(p, *oracle.moments(p, fm))) / (2 * h)
        assert np.allclose(col, J[:, j], atol=1e-7)


def test_fig2_dissipation_lowers_growth(paper_values):
    """Fig. 2: the dissipation term lowers max|omega| at every alpha."""
    for alpha in (0.1, 0.3, 0.45):
        with_d = _curve(paper_values, alpha, True).max()
        without = _curve(paper_values, alpha, False).max()
        assert with_d < without
        assert without > 1.0 + 1e-3
    assert _curve(paper_values, 0.1, True).max() <= 1.0 + 1e-12


def test_fig3_mixed_scheme_beats_upwind_at_large_dt(paper_values):
    """Fig. 3: beta = 0.25 with dissipation against beta = 0 without.  The
    former stays at max|omega| = 1 for small dt and only slightly above 1 at
    large dt; the latter is always worse and its excess grows with dt.  (The
    text's "both stable at small dt" is not reproduced: the upwind curve
    tends to 1 only as dt -> 0.)"""
    prev = 1.0
    for alpha in (0.01, 0.05, 0.1, 0.3, 0.45):
        a = _curve(paper_values, alpha, True, 0.25).max()
        b = _curve(paper_values, alpha, False, 0.0).max()
        assert a < b and b > prev
        prev = b
        if alpha <= 0.1:
            assert a <= 1.0 + 1e-12
    assert _curve(paper_values, 0.45, True, 0.25).max() < 1.02 < prev


def _max_all(paper_values, alpha, eta0=None, state=None, dx=0.01):
    """max|omega| over k along x, y and both diagonals."""
    c1, c2, e0d = paper_values["fig2_c1_c2_eta0"]
    eta0 = e0d if eta0 is None else eta0
    dt = alpha * dx / c2
    st = _fig_state(paper_values) if state is None else state
    return vn.max_growth(st, B, c1, c2, eta0, dt, dx, dt, 0.25, np.array(W.lambda_eq13(c1, dx)),
                         npts=int(paper_values["kdx_points"][0]))


def test_fig5_small_eta0_is_worst(paper_values):
    """Fig. 5 (dt = 0.3 dx / c2): eta0 = 5 is the unstable one (its growing
    modes run along y and the diagonals); 15 and 20 are nearly the same."""
    a = paper_values["fig5_alpha"][0]
    g = {e: _max_all(paper_values, a, eta0=e) for e in paper_values["fig5_eta0_values"]}
    assert g[5.0] > 1.1
    assert g[5.0] - 1.0 > 10 * (max(g[10.0], g[15.0], g[20.0]) - 1.0)
    assert abs(g[15.0] - g[20.0]) < 0.01 * (g[5.0] - 1.0)


def test_fig6_hotter_is_more_stable(paper_values):
    """Fig. 6 (dt = 0.45 dx / c2): T = 5 is more stable than T = 1.  (The
    text's further gain at T = 25 is not reproduced.)"""
    a = paper_values["fig6_alpha"][0]
    g1 = _max_all(paper_values, a, state=(1.0, 10.0, 0.0, 1.0))
    g5 = _max_all(paper_values, a, state=(1.0, 10.0, 0.0, 5.0))
    assert g5 < g1


def test_fig7_fast_flow_is_unstable(paper_values):
    """Fig. 7 (dt = 0.3 dx / c2): u1 = 15, well above c1 = 10, is clearly
    unstable and worse than any u1 <= c1."""
    a = paper_values["fig7_alpha"][0]
    g15 = _max_all(paper_values, a, state=(1.0, 15.0, 0.0, 1.0))
    slow = [_max_all(paper_values, a, state=(1.0, u, 0.0, 1.0)) for u in (0.0, 5.0, 10.0)]
    assert g15 > 1.02 and g15 - 1.0 > 4 * (max(slow) - 1.0)


def test_fig4_c2_sweep_is_singular_at_c1(paper_values):
    """Fig. 4 sweeps c2 from 10 = c1 upwards; at c2 = c1, A_i and B_i of
    Eqs. (e17), (e18) are singular."""
    with pytest.raises(ZeroDivisionError):
        vn.feq_state(1.0, 10.0, 0.0, 1.0, B, 10.0, 10.0, 10.0)


@pytest.mark.parametrize("make", [W.sod_400x4, W.ratio1000_2000x4, lambda: W.dmr(1024),
                                  W.mach3_2048x256])
def test_config_parameters_are_vetted(make):
    """Every workload's (c1, c2, eta0, alpha, lambda, beta) has max|omega| <= 1
    (to 1e-9) at the states it starts from, over k along x, y and both
    diagonals, so round-off is not amplified."""
    p = make()
    s = p.setup
    states = [s["left"], s["right"]] if s["kind"] == "riemann" else [s["pre"], s["post"]]
    for st in states:
        g = vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta, np.array(p.lam))
        assert g <= 1.0 + 1e-9, (p.name, st, g)


def test_batch_parameters_are_vetted():
    """The per-tube constants of the batched workload keep max|omega| <=
    1 + 1e-5 per step (31 wave numbers, four directions) at the left, right
    and both star states (every 8th tube of the 256)."""
    from oracle import gasdynamics as gd
    probs = W.batch_riemann()
    for p in probs[::8]:
        L, R = p.setup["left"], p.setup["right"]
        WL, WR = (L[0], L[1], L[0] * L[3]), (R[0], R[1], R[0] * R[3])
        ps, us = gd.riemann_star(WL, WR, 1.4)
        assert p.c1 > 1.05 * max(L[1], us)
        s = gd.riemann_sample(WL, WR, 1.4, [us - 1e-9, us + 1e-9])
        states = [L, R, (s[0, 0], us, 0.0, s[2, 0] / s[0, 0]), (s[0, 1], us, 0.0, s[2, 1] / s[0, 1])]
        for st in states:
            g = vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta, np.array(p.lam))
            assert g <= 1.0 + 1e-5, (p.name, st, g)


def _mach30_states():
    from oracle import gasdynamics as gd
    ps, us = gd.riemann_star((1.4, 30.0, 1.0), (1.4, 0.0, 1.0), 1.4)
    rs = gd.riemann_sample((1.4, 30.0, 1.0), (1.4, 0.0, 1.0), 1.4, [us])[0, 0]
    return [(1.4, 30.0, 0.0, 1.0 / 1.4), (1.4, 0.0, 0.0, 1.0 / 1.4), (rs, us, 0.0, ps / rs)]


@pytest.mark.parametrize("lam0", [2.0, 3.0, 4.0, 5.0])
def test_mach30_lambda0_sweep_is_vetted(lam0):
    """The Fig. 9b sweep (lambda_0 = 2..5 c1 dx, lambda_1..8 = 2 x Eq. 13,
    c1 = 33, c2 = 80, eta0 = 40, alpha = 0.05) is neutral to 1e-5 per step at
    the inflow, rest and star states of Eq. Riemann-1."""
    p = W.mach30_fig8(lam0_scale=lam0, steps=1)
    for st in _mach30_states():
        g = vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta, np.array(p.lam))
        assert g <= 1.0 + 1e-5, (lam0, st, g)


@pytest.mark.parametrize("kw", [dict(beta=0.0), dict(lam0_scale=1.0)])
def test_mach30_upwind_and_low_lambda0_grow(kw):
    """The first-order upwind scheme (beta = 0, Fig. 9a) and lambda_0 = c1 dx
    with the same constants grow by more than 2e-5 per step at the inflow
    state: these are the runs whose shock fronts go to T < 0."""
    p = W.mach30_fig8(steps=1, **kw)
    st = _mach30_states()[0]
    g = vn.max_growth(st, p.b, p.c1, p.c2, p.eta0, p.dt, p.dx, p.tau, p.beta, np.array(p.lam))
    assert g > 1.0 + 2e-5, (kw, g)
