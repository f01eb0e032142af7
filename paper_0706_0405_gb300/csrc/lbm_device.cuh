// lbm_device.cuh -- device-side pieces of the KT D2V9 finite-difference
// lattice Boltzmann step (Pan, Xu, Zhang & Jiang, IJMPC 2007) shared by the
// kernels of liblbm: the constant block, moments, equilibrium and ghost rules.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// Layout of one level in HBM: row-interleaved, [row][population][column].
// Each of the ny + 2 rows (rows 0 and ny + 1 are the ghost rows) holds the
// nine population rows of that grid row one after the other, each `pitch`
// elements long, so a node's nine values are `pitch` apart (Grid::plane) and
// consecutive grid rows 9 * pitch apart (Grid::row).  A tile of a few rows
// then lies in a few contiguous runs of HBM rather than 9 far-apart ones per
// row.  Interior column 0 sits at column PADX, so that interior row segments
// start on a 32-byte boundary for FP64 and FP32 alike; the ghost columns are
// PADX - 1 and PADX + nx.
constexpr int PADX = 4;

// Temperature recovery variants of the FP32 modes (see lbm.h).
enum TMode : int {
    T_PLAIN = 0,  // T = (E / rho - u^2) / b in the storage precision (FP64 mode)
    T_INT32 = 1,  // T = sum f_i |v_i - u|^2 (+ eta^2 on i = 0) / (b rho), FP32
    T_INT64 = 2,  // same, the nine exact FP32 products summed in FP64
    T_DF = 3,     // same, summed in double-float (error-free FP32 transforms)
    T_CONS = 4    // T = (E / rho - u^2) / b in FP32 (with the moment-exact
                  // relaxation its cancellation at high Mach only perturbs the
                  // equilibrium's non-conserved part)
};

// FP32 modes whose relaxation term is corrected to carry exactly omega times
// the mass, momentum and energy of f (see conserve below).
template <int TM>
constexpr bool moment_exact() {
    return TM == T_INT64 || TM == T_DF || TM == T_CONS;
}

enum BcKind : int { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_DIRICHLET = 2, BC_REFLECT = 3 };
enum Side : int { S_LEFT = 0, S_RIGHT = 1, S_BOTTOM = 2, S_TOP = 3 };

// Per-context constants, rounded once to the storage type on the host.
// Update of population i at node x (Eq. SEC-VON-11 with the beta-upwind
// derivative of Eqs. SEC-VON-2a/2b and central second differences folded in):
//   f_i' = w[i][0] f_i(x) + w[i][1] f_i(x+dx) + w[i][2] f_i(x-dx)
//        + w[i][3] f_i(y+dy) + w[i][4] f_i(y-dy) + omega f_i^eq(x),
// where w[i][0] already holds the 1 - omega of the identity and the
// relaxation; wi[i] = w[i][0] - (1 - omega) is the stencil's own centre
// weight, for the increment form f_i' = f_i + (stencil + relaxation
// increment) of the FP32 modes.
template <typename S>
struct Model {
    S w[9][5];
    S wi[9];
    S omega;          // dt / tau
    S c1, d;          // axis speed c1; diagonal component c2 / sqrt(2)
    S c1s, c2s, eta2; // c1^2, c2^2, eta0^2
    S inv_b;          // 1 / b
    S b;              // b = 2 / (gamma - 1)
    S k0;             // A_0 / T = (b - 2) / eta0^2 (Eq. e17)
    S a1c, a1T, a1u;  // A_1..4 = a1c + a1T T + a1u u^2 (Eq. e17)
    S a5c, a5T, a5u;  // A_5..8
    S b1c, b1T, b1u;  // B_1..4 = b1c + b1T T + b1u u^2 (Eq. e18)
    S b5c, b5T, b5u;  // B_5..8
    S D1, D5;         // D_1..4, D_5..8 (Eq. e18)
    // moment-exact relaxation (conserve): 1 / (2 c1); the set of four moving
    // populations that absorbs the mass / energy defect (0: axes 1..4,
    // 1: diagonals 5..8) with kcons = rho_o / 4 and kzero = 1 - rho_o, where
    // rho_o = (c_o^2 - eta0^2) / (c_s^2 - eta0^2) for the set's speed c_s
    // and the other set's c_o
    S h1, kcons, kzero, cons_diag;
};

// Grid and boundary description.
template <typename S>
struct Grid {
    int nx, ny, pitch;            // pitch: elements per population row (>= nx + 2 PADX)
    long long plane;              // stride between populations of a node = pitch
    long long row;                // stride between consecutive grid rows = 9 * pitch
    int kind_lo[4], kind_hi[4];
    int split_moving[4];          // 1 if split_speed != 0
    int split_index[4];           // fixed splits: first along-index in the "hi" part
    double split0[4], split_speed[4];
    double dt, dx;
    S feq[4][2][9];               // f^eq of each side's lo / hi Dirichlet state
};

// Mirror maps of a reflecting wall: reverse v_x (left/right) or v_y
// (bottom/top) of the velocities of Eq. (e14).
__host__ __device__ constexpr int mirror_x(int i) {
    return i == 1 ? 3 : i == 3 ? 1 : i == 5 ? 6 : i == 6 ? 5 : i == 7 ? 8 : i == 8 ? 7 : i;
}
__host__ __device__ constexpr int mirror_y(int i) {
    return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i;
}

// ------------------------------------------------------ explicit rounding
// Every operation of the node update is written with a round-to-nearest
// intrinsic, so the compiler cannot contract or reorder it: all kernel
// variants then produce the same bits for the same level.
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// FP32 products flush subnormal operands and results to zero (.ftz), in the
// scalar and the packed (F2) form alike: the packed product is only kept
// apart from the add or subtract that consumes it in its .ftz form (the code
// generator fuses a plain packed product into a following packed add or
// subtract, which changes the rounding), and the scalar one follows it so
// that both forms give the same bits.  Products this small never occur in
// the populations or moments of any workload.
__device__ __forceinline__ float mul_(float a, float b) {
    float r;
    asm("mul.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// FP32: the hardware approximate reciprocal (PTX rcp.approx.ftz.f32, about
// 1 ulp), issued as one instruction so that every kernel gets the same bits
// whatever it does with the result; the error of the FP32 modes is set by
// the FP32 storage of f, far above that.
__device__ __forceinline__ float rcp_(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double rcp_(double a) { return __drcp_rn(a); }
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ double neg_(double a) { return -a; }

// ------------------------------------------------- packed pairs of FP32
// F2 holds the same quantity of two nodes in one 64-bit register pair; its
// operations are the packed FP32x2 instructions of sm_100+ (add / sub / fma
// .rn.f32x2, mul .rn.ftz.f32x2), which round each lane exactly as the scalar
// operation does, so a kernel that updates two nodes with them produces the
// scalar kernels' bits with half the arithmetic instructions.  A scalar
// operand is broadcast to both lanes.
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 pair(float a, float b) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ F2 bcast(float a) { return pair(a, a); }
__device__ __forceinline__ F2 bcast(F2 a) { return a; }
__device__ __forceinline__ float2 lanes(F2 a) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
    return r;
}
__device__ __forceinline__ float lane0(F2 a) { return lanes(a).x; }
__device__ __forceinline__ float lane1(F2 a) { return lanes(a).y; }
__device__ __forceinline__ F2 add2_(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 sub2_(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 mul2_(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 fma2_(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
template <typename A, typename B>
constexpr bool any_pair = std::is_same<A, F2>::value || std::is_same<B, F2>::value;
template <typename A, typename B, typename C>
constexpr bool any_pair3 = any_pair<A, B> || std::is_same<C, F2>::value;

template <typename A, typename B, std::enable_if_t<any_pair<A, B>, int> = 0>
__device__ __forceinline__ F2 add_(A a, B b) { return add2_(bcast(a), bcast(b)); }
template <typename A, typename B, std::enable_if_t<any_pair<A, B>, int> = 0>
__device__ __forceinline__ F2 sub_(A a, B b) { return sub2_(bcast(a), bcast(b)); }
template <typename A, typename B, std::enable_if_t<any_pair<A, B>, int> = 0>
__device__ __forceinline__ F2 mul_(A a, B b) { return mul2_(bcast(a), bcast(b)); }
template <typename A, typename B, typename C, std::enable_if_t<any_pair3<A, B, C>, int> = 0>
__device__ __forceinline__ F2 fma_(A a, B b, C c) { return fma2_(bcast(a), bcast(b), bcast(c)); }
// -a exactly, subnormals and signed zeros included (there is no packed
// negation): -0 - a in each lane.
__device__ __forceinline__ F2 neg_(F2 a) { return sub2_(bcast(-0.0f), a); }
__device__ __forceinline__ F2 rcp_(F2 a) { return pair(rcp_(lane0(a)), rcp_(lane1(a))); }

// Internal energy sum_i f_i w_i with the nine exact FP32 products summed in
// FP64.
__device__ __forceinline__ float int64_energy(const float (&f)[9], const float (&w)[9]) {
    double acc = __dmul_rn((double)f[0], (double)w[0]);
#pragma unroll
    for (int i = 1; i < 9; ++i) acc = __fma_rn((double)f[i], (double)w[i], acc);
    return (float)acc;
}
// The same for two nodes: each lane's sum as above.
__device__ __forceinline__ F2 int64_energy(const F2 (&f)[9], const F2 (&w)[9]) {
    float a[9], b[9], v[9], u[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        a[i] = lane0(f[i]);
        b[i] = lane1(f[i]);
        v[i] = lane0(w[i]);
        u[i] = lane1(w[i]);
    }
    return pair(int64_energy(a, v), int64_energy(b, u));
}

// TwoSum (Knuth): s + e = a + b exactly, s = a + b rounded.
template <typename V>
__device__ __forceinline__ void two_sum(V a, V b, V& s, V& e) {
    s = add_(a, b);
    const V bb = sub_(s, a);
    e = add_(sub_(a, sub_(s, bb)), sub_(b, bb));
}

#ifndef LBM_TDF_TREE
#define LBM_TDF_TREE 0
#endif

// ---------------------------------------------------------------- moments
// rho = sum f (Eq. e4), rho u = sum f v (Eq. e5), T from Eq. (e7).
template <typename S, int TM, typename V = S>
__device__ __forceinline__ void moments(const V (&f)[9], const Model<S>& M, V& rho, V& ux, V& uy,
                                        V& T) {
    const V s14 = add_(add_(f[1], f[3]), add_(f[2], f[4]));
    const V s58 = add_(add_(f[5], f[7]), add_(f[6], f[8]));
    rho = add_(add_(f[0], s14), s58);
    const V jx = fma_(M.c1, sub_(f[3], f[1]), mul_(M.d, sub_(add_(f[6], f[7]), add_(f[5], f[8]))));
    const V jy = fma_(M.c1, sub_(f[4], f[2]), mul_(M.d, sub_(add_(f[7], f[8]), add_(f[5], f[6]))));
    const V inv = rcp_(rho);
    ux = mul_(jx, inv);
    uy = mul_(jy, inv);
    if constexpr (TM == T_PLAIN || TM == T_CONS) {
        const V E = fma_(M.eta2, f[0], fma_(M.c1s, s14, mul_(M.c2s, s58)));
        T = mul_(sub_(mul_(E, inv), fma_(ux, ux, mul_(uy, uy))), M.inv_b);
    } else {
        // Internal energy sum_i f_i (|v_i - u|^2 + eta_i^2) = E - rho u^2; its
        // terms are formed around u, so the large totals never cancel, and an
        // error in u enters only at second order.
        const V ux2 = mul_(ux, ux), uy2 = mul_(uy, uy);
        const V xm = add_(M.c1, ux), xp = sub_(M.c1, ux), ym = add_(M.c1, uy), yp = sub_(M.c1, uy);
        const V dxm = add_(M.d, ux), dxp = sub_(M.d, ux), dym = add_(M.d, uy), dyp = sub_(M.d, uy);
        const V qxm = mul_(dxm, dxm), qxp = mul_(dxp, dxp), qym = mul_(dym, dym), qyp = mul_(dyp, dyp);
        const V w[9] = {add_(M.eta2, add_(ux2, uy2)), fma_(xm, xm, uy2), fma_(ym, ym, ux2),
                        fma_(xp, xp, uy2),            fma_(yp, yp, ux2), add_(qxm, qym),
                        add_(qxp, qym),               add_(qxp, qyp),    add_(qxm, qyp)};
        V e;
        if constexpr (TM == T_INT32) {
            e = mul_(f[0], w[0]);
#pragma unroll
            for (int i = 1; i < 9; ++i) e = fma_(f[i], w[i], e);
        } else if constexpr (TM == T_INT64) {
            e = int64_energy(f, w);
        } else {  // T_DF: exact products p_i + q_i, double-float sum
#if LBM_TDF_TREE
            // the p_i summed by a tree of TwoSums (Knuth), depth 4; every
            // product and sum error collected in lo
            V p[9], q[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                p[i] = mul_(f[i], w[i]);
                q[i] = fma_(f[i], w[i], neg_(p[i]));
            }
            V s01, e01, s23, e23, s45, e45, s67, e67, s03, e03, s47, e47, s07, e07, hi, e08;
            two_sum(p[0], p[1], s01, e01);
            two_sum(p[2], p[3], s23, e23);
            two_sum(p[4], p[5], s45, e45);
            two_sum(p[6], p[7], s67, e67);
            two_sum(s01, s23, s03, e03);
            two_sum(s45, s67, s47, e47);
            two_sum(s03, s47, s07, e07);
            two_sum(s07, p[8], hi, e08);
            const V qa = add_(add_(add_(q[0], q[1]), add_(q[2], q[3])), add_(add_(q[4], q[5]), add_(q[6], q[7])));
            const V ea = add_(add_(add_(e01, e23), add_(e45, e67)), add_(add_(e03, e47), add_(e07, e08)));
            e = add_(hi, add_(add_(qa, q[8]), ea));
#elif LBM_TDF_TREE == 2
            // two sequential TwoSum chains (terms 0..4 and 5..8) merged by one
            // more TwoSum: half the dependency depth of one chain
            V ha{}, la{}, hb{}, lb{};
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                V& hi = i < 5 ? ha : hb;
                V& lo = i < 5 ? la : lb;
                const V p = mul_(f[i], w[i]);
                const V q = fma_(f[i], w[i], neg_(p));
                const V s = add_(hi, p);
                const V bb = sub_(s, hi);
                lo = add_(lo, add_(add_(sub_(hi, sub_(s, bb)), sub_(p, bb)), q));
                hi = s;
            }
            V hi, eh;
            two_sum(ha, hb, hi, eh);
            e = add_(hi, add_(add_(la, lb), eh));
#else
            // sequentially: TwoSum (Knuth) of each p_i into hi, errors in lo
            V hi{}, lo{};  // +0 in every lane
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const V p = mul_(f[i], w[i]);
                const V q = fma_(f[i], w[i], neg_(p));
                const V s = add_(hi, p);
                const V bb = sub_(s, hi);
                lo = add_(lo, add_(add_(sub_(hi, sub_(s, bb)), sub_(p, bb)), q));
                hi = s;
            }
            e = add_(hi, lo);
#endif
        }
        T = mul_(mul_(e, inv), M.inv_b);
    }
}

// Equilibrium of Eqs. (e16)-(e18) times a factor:
// fe_i = scale (A_i + B_i v.u + D_i (v.u)^2); scale = rho gives f^eq, scale =
// omega rho gives the relaxation term omega f^eq of the update directly.
template <typename S, typename V = S>
__device__ __forceinline__ void equilibrium_scaled(const Model<S>& M, V scale, V ux, V uy, V T, V (&fe)[9]) {
    const V rho = scale;
    const V u2 = fma_(ux, ux, mul_(uy, uy));
    fe[0] = mul_(rho, mul_(M.k0, T));
    // per group: rho (A + D (v.u)^2) and rho B, then fe = rho (A + D (v.u)^2) +- rho B v.u
    {  // axes, v.u = +-p (i = 3, 1), +-q (i = 4, 2)
        const V A1 = fma_(M.a1u, u2, fma_(M.a1T, T, M.a1c));
        const V B1 = fma_(M.b1u, u2, fma_(M.b1T, T, M.b1c));
        const V p = mul_(M.c1, ux), q = mul_(M.c1, uy);
        const V sp = mul_(rho, fma_(mul_(M.D1, p), p, A1)), sq = mul_(rho, fma_(mul_(M.D1, q), q, A1));
        const V rB1 = mul_(rho, B1);
        fe[1] = fma_(neg_(rB1), p, sp);
        fe[3] = fma_(rB1, p, sp);
        fe[2] = fma_(neg_(rB1), q, sq);
        fe[4] = fma_(rB1, q, sq);
    }
    {  // diagonals, v.u = +-r (i = 7, 5), +-m (i = 6, 8)
        const V A5 = fma_(M.a5u, u2, fma_(M.a5T, T, M.a5c));
        const V B5 = fma_(M.b5u, u2, fma_(M.b5T, T, M.b5c));
        const V r = mul_(M.d, add_(ux, uy)), m = mul_(M.d, sub_(ux, uy));
        const V sr = mul_(rho, fma_(mul_(M.D5, r), r, A5)), sm = mul_(rho, fma_(mul_(M.D5, m), m, A5));
        const V rB5 = mul_(rho, B5);
        fe[5] = fma_(neg_(rB5), r, sr);
        fe[7] = fma_(rB5, r, sr);
        fe[6] = fma_(rB5, m, sm);
        fe[8] = fma_(neg_(rB5), m, sm);
    }
}

template <typename S>
__device__ __forceinline__ void equilibrium(const Model<S>& M, S rho, S ux, S uy, S T, S (&fe)[9]) {
    equilibrium_scaled(M, rho, ux, uy, T, fe);
}

// omega f^eq (the relaxation term of Eq. SEC-VON-11 with omega = dt / tau).
template <typename S, typename V = S>
__device__ __forceinline__ void omega_equilibrium(const Model<S>& M, V rho, V ux, V uy, V T, V (&ofe)[9]) {
    equilibrium_scaled<S, V>(M, mul_(M.omega, rho), ux, uy, T, ofe);
}

// Moment-exact relaxation.  In FP32 the equilibrium evaluated from FP32
// moments does not carry exactly the mass, momentum and energy it was built
// from: at high Mach the internal energy is a small part of terms of size
// u^2, so each evaluation shifts T by a fixed relative amount of order
// 2^-24 u^2 / T, and the same shift recurs every step in a uniform stream (a
// drift that reaches tens of per cent over 10^4-10^5 steps at Mach 30).  The
// relaxation increments d_i = omega f^eq_i - omega f_i are formed one
// population at a time (one rounding each, so they are accurate even where
// they are tiny) and their moments are removed with the fewest populations:
//  * momentum by the opposite axis pairs (3, 1) and (4, 2):
//    d3 -= g_x, d1 += g_x with g_x = (momentum of d)_x / (2 c1) (mass and
//    |v|^2 unchanged);
//  * mass and energy by the rest population and one set of four moving
//    populations s (axes or diagonals, speed c_s, sum of v = 0): with S_s,
//    S_o the increment sums of the set and of the other set,
//    d_j += -(S_s + rho_o S_o) / 4 for the set and d_0 = -(1 - rho_o) S_o,
//    which removes mass sum d and energy sum d (|v|^2 + eta^2).
// Then d carries no mass, momentum or energy (up to its own final roundings,
// relative to the small increments), as in exact arithmetic, and the
// collision conserves them (Eqs. e4, e5, e7).
template <typename S, int TM, typename V = S>
__device__ __forceinline__ void conserve_increment(const Model<S>& M, V (&d)[9]) {
    if constexpr (moment_exact<TM>()) {
        const V sa = add_(add_(d[1], d[3]), add_(d[2], d[4]));
        const V sd = add_(add_(d[5], d[7]), add_(d[6], d[8]));
        const V djx = fma_(M.c1, sub_(d[3], d[1]), mul_(M.d, sub_(add_(d[6], d[7]), add_(d[5], d[8]))));
        const V djy = fma_(M.c1, sub_(d[4], d[2]), mul_(M.d, sub_(add_(d[7], d[8]), add_(d[5], d[6]))));
        const V gx = mul_(djx, M.h1), gy = mul_(djy, M.h1);
        if (M.cons_diag == S(0)) {
            const V t = fma_(sd, M.kcons, mul_(sa, S(0.25)));  // -delta_s
            d[0] = mul_(sd, -M.kzero);
            d[1] = sub_(add_(d[1], gx), t);
            d[3] = sub_(sub_(d[3], gx), t);
            d[2] = sub_(add_(d[2], gy), t);
            d[4] = sub_(sub_(d[4], gy), t);
        } else {
            const V t = fma_(sa, M.kcons, mul_(sd, S(0.25)));
            d[0] = mul_(sa, -M.kzero);
            d[1] = add_(d[1], gx);
            d[3] = sub_(d[3], gx);
            d[2] = add_(d[2], gy);
            d[4] = sub_(d[4], gy);
#pragma unroll
            for (int i = 5; i < 9; ++i) d[i] = sub_(d[i], t);
        }
    }
}

// The relaxation term of Eq. (SEC-VON-11) at a node, in the form update()
// takes it.  FP32 (increment form): r_i = omega (f^eq_i - f_i), moment-exact
// in the modes that ask for it.  FP64: r_i = omega f^eq_i.
template <typename S, int TM, typename V = S>
__device__ __forceinline__ void relaxation(const Model<S>& M, const V (&f)[9], V rho, V ux, V uy, V T,
                                           V (&r)[9]) {
    omega_equilibrium<S, V>(M, rho, ux, uy, T, r);
    if constexpr (std::is_same<S, float>::value) {
#pragma unroll
        for (int i = 0; i < 9; ++i) r[i] = fma_(-M.omega, f[i], r[i]);
        conserve_increment<S, TM, V>(M, r);
    }
}

// Update of one population from its five-point star and the relaxation term
// r (Eq. SEC-VON-11 with the folded weights of Model).  FP32: the paper's
// increment form, f' = c + (r + wi c + w1 e + w2 w + w3 n + w4 s): the
// increment is small next to c, so its rounding errors are too, and a node
// whose increment rounds away keeps its bits (a uniform state stays put
// instead of drifting by the roundings of a full recomputation every step).
// FP64: f' = w0 c + w1 e + w2 w + w3 n + w4 s + r.
template <typename S, typename V = S>
__device__ __forceinline__ V update(const Model<S>& M, int i, V r, V c, V e, V w, V n, V s) {
    if constexpr (std::is_same<S, float>::value) {
        V acc = fma_(M.wi[i], c, r);
        acc = fma_(M.w[i][1], e, acc);
        acc = fma_(M.w[i][2], w, acc);
        acc = fma_(M.w[i][3], n, acc);
        acc = fma_(M.w[i][4], s, acc);
        return add_(c, acc);
    } else {
        V acc = fma_(M.w[i][0], c, r);
        acc = fma_(M.w[i][1], e, acc);
        acc = fma_(M.w[i][2], w, acc);
        acc = fma_(M.w[i][3], n, acc);
        return fma_(M.w[i][4], s, acc);
    }
}

// ---------------------------------------------------------- ghost layer
// Which part (lo = 0 / hi = 1) of `side` applies at along-side coordinate
// `along` for time level `level`: lo iff along < split0 + split_speed t with
// t = level * dt, all in FP64 with explicit rounding so that the decision is
// the same as a plain IEEE evaluation of that expression on any host.
// Unsplit sides and sides with a fixed split carry the first "hi" index,
// computed on the host with the same FP64 expression; only moving splits
// (split_speed != 0) evaluate it here.
template <typename S>
__device__ __forceinline__ int side_part(const Grid<S>& G, int side, int along_index,
                                         long long level) {
    if (!G.split_moving[side]) return along_index < G.split_index[side] ? 0 : 1;
    const double t = __dmul_rn((double)level, G.dt);
    const double split = __dadd_rn(G.split0[side], __dmul_rn(G.split_speed[side], t));
    const double along = __dmul_rn((double)along_index + 0.5, G.dx);
    return along < split ? 0 : 1;
}

template <typename S>
__device__ __forceinline__ size_t cell(const Grid<S>& G, int ix, int iy) {
    return (size_t)(iy + 1) * (size_t)G.row + (size_t)(ix + PADX);
}

// Write the ghost cells of level `level` that the edge node (ix, iy), whose
// nine level values are v, is responsible for: its own side's ghost for
// OUTFLOW / REFLECT / DIRICHLET, and the opposite side's ghost for PERIODIC.
template <typename S>
__device__ __forceinline__ void write_ghosts(const Grid<S>& G, S* __restrict__ f, int ix, int iy,
                                             const S (&v)[9], long long level) {
    const size_t pl = (size_t)G.plane;
    // left / right sides: ghost columns, along-coordinate = iy
    if (ix == 0 || ix == G.nx - 1) {
#pragma unroll
        for (int side = S_LEFT; side <= S_RIGHT; ++side) {
            const int part = side_part(G, side, iy, level);
            const int kind = part ? G.kind_hi[side] : G.kind_lo[side];
            const int own = side == S_LEFT ? 0 : G.nx - 1;
            const int far = side == S_LEFT ? G.nx - 1 : 0;
            const size_t gc = (size_t)(iy + 1) * G.row + (side == S_LEFT ? PADX - 1 : PADX + G.nx);
            if (kind == BC_PERIODIC) {
                if (ix == far)
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = v[i];
            } else if (ix == own) {
                if (kind == BC_OUTFLOW)
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = v[i];
                else if (kind == BC_REFLECT)
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = v[mirror_x(i)];
                else
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = G.feq[side][part][i];
            }
        }
    }
    if (iy == 0 || iy == G.ny - 1) {
#pragma unroll
        for (int side = S_BOTTOM; side <= S_TOP; ++side) {
            const int part = side_part(G, side, ix, level);
            const int kind = part ? G.kind_hi[side] : G.kind_lo[side];
            const int own = side == S_BOTTOM ? 0 : G.ny - 1;
            const int far = side == S_BOTTOM ? G.ny - 1 : 0;
            const size_t gc = (size_t)(side == S_BOTTOM ? 0 : G.ny + 1) * G.row + (ix + PADX);
            if (kind == BC_PERIODIC) {
                if (iy == far)
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = v[i];
            } else if (iy == own) {
                if (kind == BC_OUTFLOW)
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = v[i];
                else if (kind == BC_REFLECT)
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = v[mirror_y(i)];
                else
                    for (int i = 0; i < 9; ++i) f[i * pl + gc] = G.feq[side][part][i];
            }
        }
    }
}

// Status word bits (the same values as the LBM_FLAG_* of lbm.h).
constexpr unsigned ST_NONPHYSICAL = 1u;  // rho <= 0 or a non-finite moment
constexpr unsigned ST_TIMEOUT = 2u;      // a bounded device wait gave up
constexpr unsigned ST_T_NONPOS = 4u;     // T <= 0 at some node (transient, allowed)

// Health bits of one node's moments.
// (A non-finite velocity makes T non-finite too, since T is formed from it.)
template <typename S>
__device__ __forceinline__ unsigned health(S rho, S ux, S uy, S T) {
    if (!(rho > S(0)) || !isfinite(T)) return ST_NONPHYSICAL;
    return T > S(0) ? 0u : ST_T_NONPOS;
}

// OR the bits of all active lanes into the status word with one atomic per
// warp, and only when some lane has a bit set.
__device__ __forceinline__ void report(unsigned* status, unsigned bits) {
    const unsigned m = __activemask();
    const unsigned any = __reduce_or_sync(m, bits);
    if (any && (threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicOr(status, any);
}

// ---------------------------------------------------- two nodes per thread
// Update of two x-adjacent nodes from a box in shared memory: b points at the
// first node's population 0 (8-byte aligned), populations are P floats
// apart, the rows above and below dn and ds floats away; the x neighbours
// outside the pair are b[-1] and b[2] of each population.  Writes the nine
// updated pairs to o and returns the health bits of the nodes inside the
// grid (nvalid = 1: only the first).
//
// Two forms with the same bits: both nodes at once in packed FP32x2
// arithmetic (half the arithmetic instructions, one dependency chain), or
// one after the other in scalar arithmetic (twice the instructions, two
// chains the scheduler can interleave).  Measured on the 4096 x 1024 double
// Mach reflection: packed is faster for the double-float temperature
// recovery (69.3 against 67.4 GLUPS) and the plain FP32 mode (78.9 / 77.8),
// scalar for the FP32 total-energy mode (76.8 / 68.9, where the packed form
// runs out of registers).  LBM_PAIR_PACKED: 0 scalar in every mode, 1 per
// mode as measured, 2 packed in every mode.  (The batch kernel, whose model
// constants sit in shared memory rather than in the kernel parameters, is
// faster with the scalar form in every mode: 58.0 against 54.8 GLUPS on 256
// tubes with double-float T.)
#ifndef LBM_PAIR_PACKED
#define LBM_PAIR_PACKED 1
#endif
// A pair from shared memory, read again each time (not kept in a register).
__device__ __forceinline__ F2 lds_pair(const float* p) {
    F2 r;
    asm volatile("ld.shared.b64 %0, [%1];"
                 : "=l"(r.v)
                 : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))));
    return r;
}

template <int TM>
constexpr bool packed_pair() {
    return LBM_PAIR_PACKED == 2 || (LBM_PAIR_PACKED == 1 && (TM == T_DF || TM == T_INT32));
}

// kReload (packed form): the centre pairs are read from shared memory again
// in each phase (moments, relaxation, update) instead of being kept in
// registers across all three, which lowers the register peak by 18 (so that
// more CTAs fit on an SM) for 18 more shared-memory loads.
template <int TM, bool kPacked = packed_pair<TM>(), bool kReload = false>
__device__ __forceinline__ unsigned pair_update(const Model<float>& M, const float* b, int P, int dn, int ds,
                                                int nvalid, float2 (&o)[9]) {
    unsigned bits = 0;
    if constexpr (kPacked) {
        auto centre = [&](F2 (&C)[9]) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if constexpr (kReload)
                    C[i] = lds_pair(b + i * P);
                else
                    C[i].v = *reinterpret_cast<const unsigned long long*>(b + i * P);
            }
        };
        F2 acc[9];
        {
            F2 rho, ux, uy, T;
            {
                F2 C[9];
                centre(C);
                moments<float, TM, F2>(C, M, rho, ux, uy, T);
            }
            bits |= health(lane0(rho), lane0(ux), lane0(uy), lane0(T));
            if (nvalid == 2) bits |= health(lane1(rho), lane1(ux), lane1(uy), lane1(T));
            F2 C[9];
            centre(C);
            relaxation<float, TM, F2>(M, C, rho, ux, uy, T, acc);
        }
        F2 C[9];
        centre(C);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float* bp = b + i * P;
            F2 Nn, Ss;
            Nn.v = *reinterpret_cast<const unsigned long long*>(bp + dn);
            Ss.v = *reinterpret_cast<const unsigned long long*>(bp + ds);
            const F2 Ev = pair(lane1(C[i]), bp[2]), Wv = pair(bp[-1], lane0(C[i]));
            o[i] = lanes(update<float, F2>(M, i, acc[i], C[i], Ev, Wv, Nn, Ss));
        }
    } else {
        float2 C[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) C[i] = *reinterpret_cast<const float2*>(b + i * P);
        float acc[9][2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = j ? C[i].y : C[i].x;
            float rho, ux, uy, T;
            moments<float, TM>(f, M, rho, ux, uy, T);
            if (j < nvalid) bits |= health(rho, ux, uy, T);
            float ofe[9];
            relaxation<float, TM>(M, f, rho, ux, uy, T, ofe);
#pragma unroll
            for (int i = 0; i < 9; ++i) acc[i][j] = ofe[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float* bp = b + i * P;
            const float2 Nn = *reinterpret_cast<const float2*>(bp + dn);
            const float2 Ss = *reinterpret_cast<const float2*>(bp + ds);
            const float Wv = bp[-1], Ev = bp[2];
            o[i].x = update(M, i, acc[i][0], C[i].x, C[i].y, Wv, Nn.x, Ss.x);
            o[i].y = update(M, i, acc[i][1], C[i].y, Ev, C[i].x, Nn.y, Ss.y);
        }
    }
    return bits;
}

// ------------------------------------------------------ one node per thread
// Reads the node and its four star neighbours of all nine planes (kCoherent:
// through L2 only, for data written earlier in the same kernel by other
// CTAs), updates it, writes nine values and, at an edge, the next level's
// ghost cells.  Returns the node's health bits.
template <typename S, bool kCoherent>
__device__ __forceinline__ S load_s(const S* p) {
    return kCoherent ? __ldcg(p) : __ldg(p);
}

template <typename S, int TM, bool kCoherent>
__device__ __forceinline__ unsigned node_step(const S* __restrict__ fin, S* __restrict__ fout, const Model<S>& M,
                                              const Grid<S>& G, int ix, int iy, long long level) {
    const size_t pl = (size_t)G.plane;
    const size_t c = cell(G, ix, iy);
    S f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = load_s<S, kCoherent>(fin + i * pl + c);
    S rho, ux, uy, T;
    moments<S, TM>(f, M, rho, ux, uy, T);
    const unsigned bits = health(rho, ux, uy, T);
    S ofe[9];
    relaxation<S, TM>(M, f, rho, ux, uy, T, ofe);
    S o[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const S* p = fin + i * pl + c;
        o[i] = update(M, i, ofe[i], f[i], load_s<S, kCoherent>(p + 1), load_s<S, kCoherent>(p - 1),
                      load_s<S, kCoherent>(p + G.row), load_s<S, kCoherent>(p - G.row));
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) fout[i * pl + c] = o[i];
    if (ix == 0 || iy == 0 || ix == G.nx - 1 || iy == G.ny - 1) write_ghosts(G, fout, ix, iy, o, level + 1);
    return bits;
}

// ------------------------------------------------- vectorised node group
// One thread updates V x-adjacent nodes (ix0 .. ix0 + V - 1) of row iy,
// reading the nine planes of its row segment and of the rows above and below
// as V-wide vectors and the two x-neighbours at the ends as scalars; the
// arithmetic per node is the explicitly rounded sequence of moments,
// equilibrium and update, so every kernel built on it gives the same bits.
// kCoherent: read through L2 only (data written earlier in the same kernel
// by other CTAs); otherwise through the read-only path.  Returns the health
// bits of the nodes inside the grid.
template <int V>
struct VecT;
template <>
struct VecT<2> {
    using type = float2;
};
template <>
struct VecT<4> {
    using type = float4;
};

template <int V, bool kCoherent>
__device__ __forceinline__ void load_vec(const float* p, float (&out)[V]) {
    using T = typename VecT<V>::type;
    const T v = kCoherent ? __ldcg(reinterpret_cast<const T*>(p)) : __ldg(reinterpret_cast<const T*>(p));
    if constexpr (V == 2) {
        out[0] = v.x;
        out[1] = v.y;
    } else {
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    }
}

template <int V>
__device__ __forceinline__ void store_vec(float* p, const float (&o)[V]) {
    using T = typename VecT<V>::type;
    T v;
    if constexpr (V == 2) {
        v.x = o[0];
        v.y = o[1];
    } else {
        v.x = o[0];
        v.y = o[1];
        v.z = o[2];
        v.w = o[3];
    }
    *reinterpret_cast<T*>(p) = v;
}

template <bool kCoherent>
__device__ __forceinline__ float load1(const float* p) {
    return kCoherent ? __ldcg(p) : __ldg(p);
}

template <int V, int TM, bool kCoherent>
__device__ __forceinline__ unsigned vec_group(const float* __restrict__ fin, float* __restrict__ fout,
                                              const Model<float>& M, const Grid<float>& G, int ix0, int iy,
                                              long long level) {
    const int nvalid = min(V, G.nx - ix0);  // nodes of the segment inside the grid
    const size_t pl = (size_t)G.plane;
    const size_t c0 = cell(G, ix0, iy);     // 4 V-byte aligned: ix0 + PADX is a multiple of V
    const float* in = fin + c0;

    float C[9][V];
#pragma unroll
    for (int i = 0; i < 9; ++i) load_vec<V, kCoherent>(in + i * pl, C[i]);

    float acc[9][V];  // omega f^eq, the first term of the update
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = C[i][k];
        float rho, ux, uy, T;
        moments<float, TM>(f, M, rho, ux, uy, T);
        if (k < nvalid) bits |= health(rho, ux, uy, T);
        float ofe[9];
        relaxation<float, TM>(M, f, rho, ux, uy, T, ofe);
#pragma unroll
        for (int i = 0; i < 9; ++i) acc[i][k] = ofe[i];
    }

    float* out = fout + c0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float* p = in + i * pl;
        float Nn[V], Ss[V];
        load_vec<V, kCoherent>(p + G.row, Nn);
        load_vec<V, kCoherent>(p - G.row, Ss);
        float row[V + 2];
        row[0] = load1<kCoherent>(p - 1);
        row[V + 1] = load1<kCoherent>(p + V);
#pragma unroll
        for (int k = 0; k < V; ++k) row[k + 1] = C[i][k];
        float o[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            o[k] = update(M, i, acc[i][k], row[k + 1], row[k + 2], row[k], Nn[k], Ss[k]);
        }
        if (nvalid == V) {
            store_vec<V>(out + i * pl, o);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (k < nvalid) out[i * pl + k] = o[k];
        }
    }
    // Edge nodes also write the next level's ghost cells; their nine values
    // are read back from what this thread just stored.
    const bool edge_row = iy == 0 || iy == G.ny - 1;
    if (edge_row || ix0 == 0 || ix0 + nvalid == G.nx) {
        for (int k = 0; k < nvalid; ++k) {
            const int ix = ix0 + k;
            if (!(edge_row || ix == 0 || ix == G.nx - 1)) continue;
            float v[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = out[i * pl + k];
            write_ghosts(G, fout, ix, iy, v, level + 1);
        }
    }
    return bits;
}

}  // namespace lbm
