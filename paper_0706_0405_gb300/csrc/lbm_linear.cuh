// lbm_linear.cuh -- the linearisation of the collision map f -> f^eq(q(f))
// used by the adjoint and by the von Neumann scanner: vector-Jacobian
// products of the equilibrium of Eqs. (e16)-(e18) with respect to the moments
// q = (rho, ux, uy, T), and of the moments of Eqs. (e4), (e5), (e7) with
// respect to f.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Partial derivatives of f^eq_i with respect to (rho, ux, uy, T), contracted
// with an adjoint vector a: h = sum_i a_i dF_i/dq.  With
// F_i = rho (A + B s_i + D s_i^2), s_i = v_i.u, and A, B depending on T and
// u^2 (Eqs. e16-e18), the sums over each velocity set reduce to sums and
// differences of the opposite pairs: on the axes s = -p, -q, p, q for
// i = 1..4 (p = c1 ux, q = c1 uy); on the diagonals s = -r, m, r, -m for
// i = 5..8 (r = d (ux + uy), m = d (ux - uy), d = c2 / sqrt 2).
template <typename S>
__device__ __forceinline__ void feq_vjp(const Model<S>& M, S rho, S ux, S uy, S T, const S (&a)[9],
                                                 S (&h)[4]) {
    const S u2 = ux * ux + uy * uy;
    const S A1 = M.a1c + M.a1T * T + M.a1u * u2, A5 = M.a5c + M.a5T * T + M.a5u * u2;
    const S B1 = M.b1c + M.b1T * T + M.b1u * u2, B5 = M.b5c + M.b5T * T + M.b5u * u2;
    const S p = M.c1 * ux, q = M.c1 * uy, r = M.d * (ux + uy), m = M.d * (ux - uy);
    // pair sums (P) and differences (Q, the + direction minus the - one)
    const S P13 = a[1] + a[3], Q13 = a[3] - a[1], P24 = a[2] + a[4], Q24 = a[4] - a[2];
    const S P57 = a[5] + a[7], Q57 = a[7] - a[5], P68 = a[6] + a[8], Q68 = a[6] - a[8];
    // per set: sum a, sum a s, sum a s^2
    const S Sa1 = P13 + P24, Ss1 = Q13 * p + Q24 * q, Sss1 = P13 * p * p + P24 * q * q;
    const S Sa5 = P57 + P68, Ss5 = Q57 * r + Q68 * m, Sss5 = P57 * r * r + P68 * m * m;
    // sum a v_x, sum a v_y and sum a s v_x, sum a s v_y per set
    const S Svx1 = M.c1 * Q13, Svy1 = M.c1 * Q24;
    const S Ssvx1 = M.c1 * p * P13, Ssvy1 = M.c1 * q * P24;
    const S Svx5 = M.d * (Q57 + Q68), Svy5 = M.d * (Q57 - Q68);
    const S Ssvx5 = M.d * (r * P57 + m * P68), Ssvy5 = M.d * (r * P57 - m * P68);
    h[0] = a[0] * (M.k0 * T) + (A1 * Sa1 + B1 * Ss1 + M.D1 * Sss1) + (A5 * Sa5 + B5 * Ss5 + M.D5 * Sss5);
    // d/du: rho [2 (A_u + B_u s) u + (B + 2 D s) v] summed with a
    const S G1 = S(2) * (M.a1u * Sa1 + M.b1u * Ss1), G5 = S(2) * (M.a5u * Sa5 + M.b5u * Ss5);
    h[1] = rho * ((G1 + G5) * ux + B1 * Svx1 + S(2) * M.D1 * Ssvx1 + B5 * Svx5 + S(2) * M.D5 * Ssvx5);
    h[2] = rho * ((G1 + G5) * uy + B1 * Svy1 + S(2) * M.D1 * Ssvy1 + B5 * Svy5 + S(2) * M.D5 * Ssvy5);
    h[3] = rho * (a[0] * M.k0 + M.a1T * Sa1 + M.b1T * Ss1 + M.a5T * Sa5 + M.b5T * Ss5);
}

// g_j = sum_m h_m dq_m/df_j at moments (rho, ux, uy, T):
// drho/df_j = 1, du/df_j = (v_j - u) / rho, dT/df_j = (|v_j - u|^2 + eta_j^2 - b T) / (b rho).
// Expanding |v_j - u|^2 with H = (h_ux, h_uy) / rho and H3 = h_T / (b rho):
// g_j = G0 + v_j.(X, Y) + H3 (|v_j|^2 + eta_j^2), where (X, Y) = H - 2 H3 u and
// G0 = h_rho - H.u + H3 (u^2 - b T); each velocity set then needs one product
// per direction.
template <typename S>
__device__ __forceinline__ void moments_vjp(const Model<S>& M, S rho, S ux, S uy, S T, const S (&h)[4],
                                            S (&g)[9]) {
    const S ir = rcp_(rho);
    const S H1 = h[1] * ir, H2 = h[2] * ir, H3 = h[3] * ir * M.inv_b;
    const S G0 = h[0] - H1 * ux - H2 * uy + H3 * (ux * ux + uy * uy - M.b * T);
    const S X = H1 - S(2) * H3 * ux, Y = H2 - S(2) * H3 * uy;
    const S g1 = G0 + H3 * M.c1s, g5 = G0 + H3 * M.c2s;
    const S cx = M.c1 * X, cy = M.c1 * Y, dp = M.d * (X + Y), dm = M.d * (X - Y);
    g[0] = G0 + H3 * M.eta2;
    g[1] = g1 - cx;
    g[2] = g1 - cy;
    g[3] = g1 + cx;
    g[4] = g1 + cy;
    g[5] = g5 - dp;
    g[6] = g5 + dm;
    g[7] = g5 + dp;
    g[8] = g5 - dm;
}

}  // namespace lbm
