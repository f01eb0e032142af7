// lbm_linear.cuh -- the linearisation of the collision map f -> f^eq(q(f))
// used by the adjoint and by the von Neumann scanner: vector-Jacobian
// products of the equilibrium of Eqs. (e16)-(e18) with respect to the moments
// q = (rho, ux, uy, T), and of the moments of Eqs. (e4), (e5), (e7) with
// respect to f.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Partial derivatives of f^eq_i with respect to (rho, ux, uy, T), contracted
// with an adjoint vector a: h = sum_i a_i dF_i/dq.
template <typename S>
__host__ __device__ __forceinline__ void feq_vjp(const Model<S>& M, S rho, S ux, S uy, S T, const S (&a)[9],
                                        S (&h)[4]) {
    const S u2 = ux * ux + uy * uy;
    const S A1 = M.a1c + M.a1T * T + M.a1u * u2, A5 = M.a5c + M.a5T * T + M.a5u * u2;
    const S B1 = M.b1c + M.b1T * T + M.b1u * u2, B5 = M.b5c + M.b5T * T + M.b5u * u2;
    const int sx[9] = {0, -1, 0, 1, 0, -1, 1, 1, -1};
    const int sy[9] = {0, 0, -1, 0, 1, -1, -1, 1, 1};
    S hr = a[0] * (M.k0 * T), hx = S(0), hy = S(0), hT = a[0] * (rho * M.k0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const bool axis = i <= 4;
        const S mag = axis ? M.c1 : M.d;
        const S vx = sx[i] * mag, vy = sy[i] * mag;
        const S A = axis ? A1 : A5, B = axis ? B1 : B5, D = axis ? M.D1 : M.D5;
        const S Au = axis ? M.a1u : M.a5u, Bu = axis ? M.b1u : M.b5u;
        const S AT = axis ? M.a1T : M.a5T, BT = axis ? M.b1T : M.b5T;
        const S vu = vx * ux + vy * uy;
        hr += a[i] * (A + B * vu + D * vu * vu);
        const S g = S(2) * (Au + Bu * vu);   // d(A + B v.u)/d(u^2) * 2
        const S k = B + S(2) * D * vu;        // d(B v.u + D (v.u)^2)/d(v.u)
        hx += a[i] * rho * (g * ux + k * vx);
        hy += a[i] * rho * (g * uy + k * vy);
        hT += a[i] * rho * (AT + BT * vu);
    }
    h[0] = hr;
    h[1] = hx;
    h[2] = hy;
    h[3] = hT;
}

// g_j = sum_m h_m dq_m/df_j at moments (rho, ux, uy, T):
// drho/df_j = 1, du/df_j = (v_j - u) / rho, dT/df_j = (|v_j - u|^2 + eta_j^2 - b T) / (b rho).
template <typename S>
__host__ __device__ __forceinline__ void moments_vjp(const Model<S>& M, S rho, S ux, S uy, S T, const S (&h)[4],
                                            S (&g)[9]) {
    const int sx[9] = {0, -1, 0, 1, 0, -1, 1, 1, -1};
    const int sy[9] = {0, 0, -1, 0, 1, -1, -1, 1, 1};
    const S ir = S(1) / rho;
    const S b = S(1) / M.inv_b;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const S mag = j == 0 ? S(0) : (j <= 4 ? M.c1 : M.d);
        const S dx = sx[j] * mag - ux, dy = sy[j] * mag - uy;
        const S e2 = j == 0 ? M.eta2 : S(0);
        g[j] = h[0] + (h[1] * dx + h[2] * dy) * ir + h[3] * (dx * dx + dy * dy + e2 - b * T) * ir * M.inv_b;
    }
}

}  // namespace lbm
