"""von Neumann amplification matrix of the scheme (Sec. 3 of the paper).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

A small perturbation F_i exp(i k.x) of a uniform state f^0 = f^eq(rho, u, T)
is advanced by one step of Eq. (SEC-VON-11) as F^{t+dt} = G F^t with

    G_ij = (1 - w) delta_ij + w d f_i^eq / d f_j
           - (dt / dx) sum_a v_ia phi_a(k_a dx) delta_ij
           - lambda_i (dt / dx^2) sum_a (2 - 2 cos(k_a dx)) delta_ij,

w = dt / tau.  With w = 1 this is Eq. (SEC-VON-12); the (1 - w) delta term is
the one of Eq. (SEC-VON-8).  phi is Eq. (SEC-VON-9):

    v >= 0:  phi = beta e^{i th} + (1 - 2 beta) - (1 - beta) e^{-i th}
    v <  0:  phi = (1 - beta) e^{i th} - (1 - 2 beta) - beta e^{-i th}.

d f^eq / d f is the Jacobian of f -> f^eq(moments(f)) at f^0 (Eqs. e4, e5,
e7, e16-e18).  It is taken by complex-step differentiation, which is exact to
round-off for this rational map, so no hand-derived chain rule enters.
"""
from __future__ import annotations

import numpy as np

# Direction signs of Eq. (e14) (diagonals read as c2 (cos th, sin th)).
SX = np.array([0, -1, 0, 1, 0, -1, 1, 1, -1])
SY = np.array([0, 0, -1, 0, 1, -1, -1, 1, 1])


def velocities(c1: float, c2: float):
    """Eq. (e14)."""
    mag = np.array([0.0] + [c1] * 4 + [c2 / np.sqrt(2.0)] * 4)
    return SX * mag, SY * mag


def feq_state(rho, ux, uy, T, b, c1, c2, eta0):
    """Eqs. (e16)-(e18) with A_0 = (b - 2) T / eta0^2; complex inputs allowed."""
    vx, vy = velocities(c1, c2)
    c1s, c2s, e0s = c1 * c1, c2 * c2, eta0 * eta0
    u2 = ux * ux + uy * uy
    A0 = (b - 2.0) * T / e0s
    A1 = (-c2s + ((b - 2.0) * c2s / e0s + 2.0) * T + c2s / c1s * u2) / (4.0 * (c1s - c2s))
    A5 = (-c1s + ((b - 2.0) * c1s / e0s + 2.0) * T + c1s / c2s * u2) / (4.0 * (c2s - c1s))
    B1 = (-c2s + (b + 2.0) * T + u2) / (2.0 * c1s * (c1s - c2s))
    B5 = (-c1s + (b + 2.0) * T + u2) / (2.0 * c2s * (c2s - c1s))
    D1 = 1.0 / (2.0 * c1s * c1s)
    D5 = 1.0 / (2.0 * c2s * c2s)
    out = []
    for i in range(9):
        vu = vx[i] * ux + vy[i] * uy
        if i == 0:
            out.append(rho * A0)
        elif i <= 4:
            out.append(rho * (A1 + B1 * vu + D1 * vu * vu))
        else:
            out.append(rho * (A5 + B5 * vu + D5 * vu * vu))
    return np.array(out)


def moments_of(f, b, c1, c2, eta0):
    """Eqs. (e4), (e5), (e7): (rho, ux, uy, T); complex inputs allowed."""
    vx, vy = velocities(c1, c2)
    eta2 = np.array([eta0 * eta0] + [0.0] * 8)
    rho = np.sum(f)
    ux = np.sum(f * vx) / rho
    uy = np.sum(f * vy) / rho
    E = np.sum(f * (vx * vx + vy * vy + eta2))
    T = (E / rho - (ux * ux + uy * uy)) / b
    return rho, ux, uy, T


def feq_jacobian(state, b, c1, c2, eta0, h: float = 1e-30) -> np.ndarray:
    """J_ij = d f_i^eq / d f_j at f = f^eq(state), by complex step."""
    rho, ux, uy, T = state
    f0 = feq_state(rho, ux, uy, T, b, c1, c2, eta0).astype(complex)
    J = np.zeros((9, 9))
    for j in range(9):
        fp = f0.copy()
        fp[j] += 1j * h
        J[:, j] = np.imag(feq_state(*moments_of(fp, b, c1, c2, eta0), b, c1, c2, eta0)) / h
    return J


def phi(theta: float, sign: int, beta: float) -> complex:
    """Eq. (SEC-VON-9) for one axis; sign = sign of v_ia (0 counts as >= 0)."""
    e = np.exp(1j * theta)
    if sign >= 0:
        return beta * e + (1.0 - 2.0 * beta) - (1.0 - beta) / e
    return (1.0 - beta) * e - (1.0 - 2.0 * beta) - beta / e


def amplification_matrix(kxdx, kydx, state, b, c1, c2, eta0, dt, dx, tau, beta, lam, J=None):
    """G(k) of Eqs. (SEC-VON-8, 12) for the wave vector (kx dx, ky dx)."""
    vx, vy = velocities(c1, c2)
    w = dt / tau
    if J is None:
        J = feq_jacobian(state, b, c1, c2, eta0)
    G = w * J.astype(complex) + (1.0 - w) * np.eye(9)
    for i in range(9):
        adv = vx[i] * phi(kxdx, SX[i], beta) + vy[i] * phi(kydx, SY[i], beta)
        diss = lam[i] * ((2.0 - 2.0 * np.cos(kxdx)) + (2.0 - 2.0 * np.cos(kydx)))
        G[i, i] -= (dt / dx) * adv + (dt / dx ** 2) * diss
    return G


def spectral_radius(G: np.ndarray) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(G))))


def growth_curve(state, b, c1, c2, eta0, dt, dx, tau, beta, lam, direction=(1, 0), npts=31):
    """max|omega| at kdx = 0 .. pi in npts points (the paper uses 31 points,
    k along x) for the wave direction (dx, dy) in {(1,0), (0,1), (1,1), (1,-1)}."""
    J = feq_jacobian(state, b, c1, c2, eta0)
    th = np.linspace(0.0, np.pi, npts)
    return th, np.array([
        spectral_radius(amplification_matrix(direction[0] * t, direction[1] * t, state, b, c1,
                                             c2, eta0, dt, dx, tau, beta, lam, J))
        for t in th
    ])


def max_growth(state, b, c1, c2, eta0, dt, dx, tau, beta, lam, npts=31,
               directions=((1, 0), (0, 1), (1, 1), (1, -1))) -> float:
    """Largest max|omega| over the listed wave directions."""
    return max(float(np.max(growth_curve(state, b, c1, c2, eta0, dt, dx, tau, beta, lam, d,
                                         npts)[1])) for d in directions)
