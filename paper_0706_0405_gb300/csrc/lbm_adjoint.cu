// lbm_adjoint.cu -- the hand-written adjoint of the fused step: the transpose
// of the linearised update of Eq. (SEC-VON-11) (transposed five-point star,
// ghost links through the boundary rule, transposed collision Jacobian), the
// tau derivative, and the vector-Jacobian products of the equilibrium
// (Eqs. e16-e18) and of the moments (Eqs. e4, e5, e7).
#include "lbm_launch.h"
#include "lbm_linear.cuh"
#include "lbm_ptx.cuh"

namespace lbm {

namespace {
constexpr int kThreads = 256;

inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

template <typename S>
__device__ __forceinline__ int kind_at(const Grid<S>& G, int side, int along_index, long long level) {
    return side_part(G, side, along_index, level) ? G.kind_hi[side] : G.kind_lo[side];
}

// Adjoint of one node (gather form over the transposed star): from f at the
// node (fv), the adjoint of level n + 1 at the node (av) and at its four star
// neighbours (aL, aR, aD, aU; zero where the star leaves the grid through a
// non-periodic side), the adjoint of level n at the node (o) before the ghost
// links, and the node's tau term tn = sum_i a_i (f^eq_i - f_i).  Both adjoint
// kernels use it, so they round alike.
// The collision part: g = (df^eq/df)^T a at the node (through the moments)
// and the tau term tn.
template <typename S, int TM>
__device__ __forceinline__ void adjoint_collision(const Model<S>& M, const S (&fv)[9], const S (&av)[9],
                                                  S (&g)[9], S& tn) {
    S rho, ux, uy, T;
    moments<S, TM>(fv, M, rho, ux, uy, T);
    S h[4];
    feq_vjp(M, rho, ux, uy, T, av, h);
    // tau term: f^eq is linear in rho, so sum_i a_i f^eq_i = rho dF/drho . a
    // = rho h[0]; no equilibrium needs evaluating
    S af = mul_(av[0], fv[0]);
#pragma unroll
    for (int i = 1; i < 9; ++i) af = fma_(av[i], fv[i], af);
    tn = fma_(rho, h[0], neg_(af));
    moments_vjp(M, rho, ux, uy, T, h, g);
}

// Adjoint of population j of one node from the transposed star: its own
// weight with the collision term, then the nodes left of, right of, below
// and above it, which read it as their E, W, N and S neighbour.
template <typename S>
__device__ __forceinline__ S adjoint_star(const Model<S>& M, int j, S g, S a, S aL, S aR, S aD, S aU) {
    S r = fma_(M.w[j][0], a, mul_(M.omega, g));
    r = fma_(M.w[j][1], aL, r);
    r = fma_(M.w[j][2], aR, r);
    r = fma_(M.w[j][3], aD, r);
    return fma_(M.w[j][4], aU, r);
}

template <typename S, int TM>
__device__ __forceinline__ void adjoint_core(const Model<S>& M, const S (&fv)[9], const S (&av)[9],
                                             const S (&aL)[9], const S (&aR)[9], const S (&aD)[9],
                                             const S (&aU)[9], S (&o)[9], S& tn) {
    S g[9];
    adjoint_collision<S, TM>(M, fv, av, g, tn);
#pragma unroll
    for (int j = 0; j < 9; ++j) o[j] = adjoint_star(M, j, g[j], av[j], aL[j], aR[j], aD[j], aU[j]);
}

// Ghost links of an edge node: its own ghost cell on a non-periodic side is
// made from it (outflow: copied; reflect: mirrored), so the weight that read
// that ghost comes back to it.  Dirichlet ghosts depend on nothing.
template <typename S>
__device__ __forceinline__ void adjoint_ghost_links(const Model<S>& M, const Grid<S>& G, long long level,
                                                    int ix, int iy, const S (&av)[9], S (&o)[9]) {
    const int kl = ix == 0 ? kind_at(G, S_LEFT, iy, level) : -1;
    const int kr = ix == G.nx - 1 ? kind_at(G, S_RIGHT, iy, level) : -1;
    const int kb = iy == 0 ? kind_at(G, S_BOTTOM, ix, level) : -1;
    const int kt = iy == G.ny - 1 ? kind_at(G, S_TOP, ix, level) : -1;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        S r = o[j];
        if (kl == BC_OUTFLOW) r = fma_(M.w[j][2], av[j], r);
        if (kl == BC_REFLECT) r = fma_(M.w[mirror_x(j)][2], av[mirror_x(j)], r);
        if (kr == BC_OUTFLOW) r = fma_(M.w[j][1], av[j], r);
        if (kr == BC_REFLECT) r = fma_(M.w[mirror_x(j)][1], av[mirror_x(j)], r);
        if (kb == BC_OUTFLOW) r = fma_(M.w[j][4], av[j], r);
        if (kb == BC_REFLECT) r = fma_(M.w[mirror_y(j)][4], av[mirror_y(j)], r);
        if (kt == BC_OUTFLOW) r = fma_(M.w[j][3], av[j], r);
        if (kt == BC_REFLECT) r = fma_(M.w[mirror_y(j)][3], av[mirror_y(j)], r);
        o[j] = r;
    }
}

// Periodic ghost cells of an adjoint level (the tile adjoint reads the star
// of every node from a box that includes the ghost layer; ghost cells of
// non-periodic sides stay zero).  Written by the node whose value wraps.
template <typename S>
__device__ __forceinline__ void write_periodic_ghosts(const Grid<S>& G, S* __restrict__ a, int ix, int iy,
                                                      const S (&v)[9]) {
    const size_t pl = (size_t)G.plane;
    if (G.kind_lo[S_LEFT] == BC_PERIODIC) {
        if (ix == G.nx - 1)
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i * pl + (size_t)(iy + 1) * G.row + (PADX - 1)] = v[i];
        if (ix == 0)
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i * pl + (size_t)(iy + 1) * G.row + (PADX + G.nx)] = v[i];
    }
    if (G.kind_lo[S_BOTTOM] == BC_PERIODIC) {
        if (iy == G.ny - 1)
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i * pl + (size_t)ix + PADX] = v[i];
        if (iy == 0)
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i * pl + (size_t)(G.ny + 1) * G.row + ix + PADX] = v[i];
    }
}

// Star neighbours of node (ix, iy) on the grid, with periodic wrap; -1 if
// none (a non-periodic edge).
template <typename S>
__device__ __forceinline__ void star_neighbours(const Grid<S>& G, int ix, int iy, int& xl, int& xr, int& yd,
                                                int& yu) {
    const bool perx = G.kind_lo[S_LEFT] == BC_PERIODIC;
    const bool pery = G.kind_lo[S_BOTTOM] == BC_PERIODIC;
    xl = ix > 0 ? ix - 1 : (perx ? G.nx - 1 : -1);
    xr = ix < G.nx - 1 ? ix + 1 : (perx ? 0 : -1);
    yd = iy > 0 ? iy - 1 : (pery ? G.ny - 1 : -1);
    yu = iy < G.ny - 1 ? iy + 1 : (pery ? 0 : -1);
}

// One adjoint step from level n + 1 back to level n, one thread per node.
// a: adjoint of level n + 1, abar: adjoint of level n (interior of the
// padded layout; ghost cells are never read or written).
// taup[block] += sum over the block's nodes of the node tau terms (per node
// in the storage precision, across nodes in FP64; the tau derivative is
// -(dt / tau^2) times the total).
template <typename S, int TM>
__global__ void __launch_bounds__(kThreads) k_adjoint(const S* __restrict__ f, const S* __restrict__ a,
                                                      S* __restrict__ abar, const Model<S> M,
                                                      const Grid<S> G, long long level,
                                                      double* __restrict__ taup) {
    __shared__ double sh[kThreads / 32];
    const long long n = (long long)G.nx * G.ny;
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    S tsum = S(0);
    if (q < n) {
        const int iy = (int)(q / G.nx), ix = (int)(q % G.nx);
        const size_t pl = (size_t)G.plane;
        const size_t c = cell(G, ix, iy);
        int xl, xr, yd, yu;
        star_neighbours(G, ix, iy, xl, xr, yd, yu);
        S fv[9], av[9], aL[9], aR[9], aD[9], aU[9], o[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fv[i] = f[i * pl + c];
            av[i] = a[i * pl + c];
            aL[i] = xl >= 0 ? a[i * pl + cell(G, xl, iy)] : S(0);
            aR[i] = xr >= 0 ? a[i * pl + cell(G, xr, iy)] : S(0);
            aD[i] = yd >= 0 ? a[i * pl + cell(G, ix, yd)] : S(0);
            aU[i] = yu >= 0 ? a[i * pl + cell(G, ix, yu)] : S(0);
        }
        adjoint_core<S, TM>(M, fv, av, aL, aR, aD, aU, o, tsum);
        if (ix == 0 || iy == 0 || ix == G.nx - 1 || iy == G.ny - 1)
            adjoint_ghost_links(M, G, level, ix, iy, av, o);
#pragma unroll
        for (int j = 0; j < 9; ++j) abar[j * pl + c] = o[j];
    }
    // warp sums in the storage precision (fixed shuffle tree), then the
    // block's eight warp sums in FP64 in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(0xffffffffu, tsum, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x / 32] = (double)tsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
        taup[blockIdx.x] += t;
    }
}

// Periodic ghost cells of an adjoint level written by something other than
// an adjoint kernel (the caller's adjoint, unpacked).
__global__ void k_adjoint_wrap(float* __restrict__ a, const Grid<float> G) {
    const long long n = (long long)G.nx * G.ny;
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (q >= n) return;
    const int iy = (int)(q / G.nx), ix = (int)(q % G.nx);
    if (!(ix == 0 || iy == 0 || ix == G.nx - 1 || iy == G.ny - 1)) return;
    float v[9];
    const size_t c = cell(G, ix, iy);
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = a[i * (size_t)G.plane + c];
    write_periodic_ghosts(G, a, ix, iy, v);
}

// ------------------------------------------------------ FP32 tile adjoint
// Persistent CTAs of 64 x 4 threads walk 64 x 4-node tiles, one node per
// thread.  Per tile one thread issues two tiled tensor copies into one of two
// shared-memory stages, completing on the stage's mbarrier: the adjoint of
// level n + 1 over the tile and its halo (72 x 6 x 9; 4 extra columns each
// side keep the x coordinate 16-byte aligned) and f of level n over the tile
// (64 x 4 x 9).  Star neighbours come from shared memory; across a periodic
// edge they come from the level's ghost cells, which the kernel that wrote
// the level filled (write_periodic_ghosts).  One thread waits (bounded; on
// give-up the CTA raises ST_TIMEOUT, drains its copies and returns) while the
// others sleep in the barrier, which also frees the previous stage.
#ifndef LBM_ADJ_TY
#define LBM_ADJ_TY 4
#endif
#ifndef LBM_ADJ_NPT
#define LBM_ADJ_NPT 1
#endif
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS (LBM_ADJ_NPT == 2 ? 4 : 3)
#endif
constexpr int kAdjTX = 64, kAdjTY = LBM_ADJ_TY, kAdjNpt = LBM_ADJ_NPT;
constexpr int kAdjThreads = kAdjTX / kAdjNpt * kAdjTY;  // kAdjNpt x-adjacent nodes per thread
constexpr int kAdjBoxX = kAdjTX + 8, kAdjBoxY = kAdjTY + 2;
constexpr int kAdjAFloats = kAdjBoxX * kAdjBoxY * 9;
constexpr int kAdjAPad = (kAdjAFloats + 31) / 32 * 32;  // the f box starts on a 128-byte boundary
constexpr int kAdjFFloats = kAdjTX * kAdjTY * 9;
constexpr int kAdjStageFloats = (kAdjAPad + kAdjFFloats + 31) / 32 * 32;
constexpr size_t kAdjSmem = 128 + sizeof(float) * 2 * kAdjStageFloats + 2 * sizeof(uint64_t);
constexpr uint32_t kAdjWaitLimit = 1u << 22;

template <int TM>
__global__ void __launch_bounds__(kAdjThreads, LBM_ADJ_MIN_BLOCKS)
    k_adjoint_tile(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapF,
                   float* __restrict__ abar, const Model<float> M,
                   const Grid<float> G, long long level, double* __restrict__ taup, int tiles_x, int ntiles,
                   unsigned* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    float* stage0 = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(float) * 2 * kAdjStageFloats);
    __shared__ int abort_flag;
    __shared__ double wsum_sh[kAdjThreads / 32];
    constexpr int kLanesX = kAdjTX / kAdjNpt;
    const int tid = threadIdx.x, tx = tid % kLanesX, ty = tid / kLanesX;
    // launched as a programmatic dependent of the previous adjoint step: no
    // level, adjoint level or tau slot is touched before that grid is done
    grid_dependency_wait();
    grid_dependents_launch();
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    auto issue = [&](int tile, int st) {
        const int x0 = (tile % tiles_x) * kAdjTX, y0 = (tile / tiles_x) * kAdjTY;
        float* dst = stage0 + st * kAdjStageFloats;
        mbar_arrive_expect_tx(&bar[st], (uint32_t)(sizeof(float) * (kAdjAFloats + kAdjFFloats)));
        // adjoint box: array column x0 = interior x0 - 4, array row y0 = interior y0 - 1
        tma_load_3d(dst, &tmapA, x0, 0, y0, &bar[st]);
        // f box: the tile itself (array column x0 + 4, row y0 + 1)
        tma_load_3d(dst + kAdjAPad, &tmapF, x0 + PADX, 0, y0 + 1, &bar[st]);
    };
    auto wait = [&](int k) { return mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), kAdjWaitLimit); };
    int issued = -1, waited = -1;
    if (blockIdx.x < ntiles) {
        if (tid == 0) issue(blockIdx.x, 0);
        issued = 0;
    }
    const size_t pl = (size_t)G.plane;
    // boxes in shared memory are [row][population][column], like the levels:
    // population strides PA, PF and row strides RA, RF
    constexpr int PA = kAdjBoxX, RA = 9 * kAdjBoxX, PF = kAdjTX, RF = 9 * kAdjTX;
    float wsum = 0.0f;  // this warp's tau terms, tile by tile in a fixed order (FP32 over a few tiles)
    // tile coordinates walked incrementally (t advances by gridDim.x): no
    // integer division per tile
    const int step_x = (int)gridDim.x % tiles_x, step_y = (int)gridDim.x / tiles_x;
    int tile_x = (int)blockIdx.x % tiles_x, tile_y = (int)blockIdx.x / tiles_x;
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        if (k > 0) {
            tile_x += step_x;
            tile_y += step_y;
            if (tile_x >= tiles_x) {
                tile_x -= tiles_x;
                ++tile_y;
            }
        }
        if (tid == 0 && !wait(k)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) {
            for (int j = waited + 1; j <= issued; ++j) wait(j);
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        waited = k;
        if (t + (int)gridDim.x < ntiles) {
            if (tid == 0) issue(t + gridDim.x, (k + 1) & 1);
            issued = k + 1;
        }
        float tn = 0.0f;
        if constexpr (kAdjNpt == 1) {
            const int ix = tile_x * kAdjTX + tx, iy = tile_y * kAdjTY + ty;
            if (ix < G.nx && iy < G.ny) {
                const float* sA = stage0 + (k & 1) * kAdjStageFloats + (ty + 1) * RA + (tx + 4);
                const float* sF = stage0 + (k & 1) * kAdjStageFloats + kAdjAPad + ty * RF + tx;
                // the box holds the star of every node: interior neighbours, the
                // wrapped values in the ghost cells of periodic sides, zeros in
                // the ghost cells of the others
                float fv[9], av[9], aL[9], aR[9], aD[9], aU[9], o[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float* pA = sA + i * PA;
                    fv[i] = sF[i * PF];
                    av[i] = pA[0];
                    aL[i] = pA[-1];
                    aR[i] = pA[1];
                    aD[i] = pA[-RA];
                    aU[i] = pA[RA];
                }
                adjoint_core<float, TM>(M, fv, av, aL, aR, aD, aU, o, tn);
                const size_t c = cell(G, ix, iy);
                if (ix == 0 || iy == 0 || ix == G.nx - 1 || iy == G.ny - 1) {
                    adjoint_ghost_links(M, G, level, ix, iy, av, o);
                    write_periodic_ghosts(G, abar, ix, iy, o);
                }
#pragma unroll
                for (int j = 0; j < 9; ++j) abar[j * pl + c] = o[j];
            }
        } else {  // two x-adjacent nodes per thread: 8-byte shared loads and stores
            const int ix0 = tile_x * kAdjTX + 2 * tx, iy = tile_y * kAdjTY + ty;
            if (ix0 < G.nx && iy < G.ny) {
                const int nvalid = min(2, G.nx - ix0);
                const float* sA = stage0 + (k & 1) * kAdjStageFloats + (ty + 1) * RA + (2 * tx + 4);
                const float* sF = stage0 + (k & 1) * kAdjStageFloats + kAdjAPad + ty * RF + 2 * tx;
                float2 A2[9];
                float g[2][9];
                float tt[2];
#pragma unroll
                for (int i = 0; i < 9; ++i) A2[i] = *reinterpret_cast<const float2*>(sA + i * PA);
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    float fv[9], av[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        fv[i] = sF[i * PF + n];
                        av[i] = n ? A2[i].y : A2[i].x;
                    }
                    adjoint_collision<float, TM>(M, fv, av, g[n], tt[n]);
                }
                // a node past the right edge (odd nx) has f = 0 in the box:
                // its terms are not used
                tn = nvalid == 2 ? add_(tt[0], tt[1]) : tt[0];
                float o[2][9];
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const float* pA = sA + j * PA;
                    const float2 Nn = *reinterpret_cast<const float2*>(pA + RA);
                    const float2 Ss = *reinterpret_cast<const float2*>(pA - RA);
                    const float Wv = pA[-1], Ev = pA[2];
                    o[0][j] = adjoint_star(M, j, g[0][j], A2[j].x, Wv, A2[j].y, Ss.x, Nn.x);
                    o[1][j] = adjoint_star(M, j, g[1][j], A2[j].y, A2[j].x, Ev, Ss.y, Nn.y);
                }
                float* out = abar + cell(G, ix0, iy);  // 8-byte aligned: ix0 + PADX is even
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    if (nvalid == 2)
                        *reinterpret_cast<float2*>(out + j * pl) = make_float2(o[0][j], o[1][j]);
                    else
                        out[j * pl] = o[0][j];
                }
                // edge nodes: the ghost links, on the values just stored (read
                // back) and the node's adjoint from the box
                const bool edge_row = iy == 0 || iy == G.ny - 1;
                if (edge_row || ix0 == 0 || ix0 + nvalid == G.nx) {
#pragma unroll 1
                    for (int n = 0; n < nvalid; ++n) {
                        const int ix = ix0 + n;
                        if (!(edge_row || ix == 0 || ix == G.nx - 1)) continue;
                        float av[9], on[9];
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            av[i] = sA[i * PA + n];
                            on[i] = out[i * pl + n];
                        }
                        adjoint_ghost_links(M, G, level, ix, iy, av, on);
                        write_periodic_ghosts(G, abar, ix, iy, on);
#pragma unroll
                        for (int i = 0; i < 9; ++i) out[i * pl + n] = on[i];
                    }
                }
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) tn += __shfl_down_sync(0xffffffffu, tn, s);
        wsum += tn;  // lane 0 holds the warp's sum
    }
    if ((tid & 31) == 0) wsum_sh[tid / 32] = (double)wsum;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) tot += wsum_sh[w];
        taup[blockIdx.x] += tot;
    }
}

// Seed: abar_j = sum_m qbar_m dq_m/df_j at the level f (qbar may have null
// components = zero); dense output.
template <typename S, int TM>
__global__ void k_moments_vjp(const S* __restrict__ f, const S* __restrict__ qr, const S* __restrict__ qx,
                              const S* __restrict__ qy, const S* __restrict__ qT, S* __restrict__ abar,
                              const Model<S> M, const Grid<S> G) {
    const long long n = (long long)G.nx * G.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(q / G.nx), ix = (int)(q % G.nx);
        const size_t c = cell(G, ix, iy);
        S fv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fv[i] = f[i * (size_t)G.plane + c];
        S rho, ux, uy, T;
        moments<S, TM>(fv, M, rho, ux, uy, T);
        const S h[4] = {qr ? qr[q] : S(0), qx ? qx[q] : S(0), qy ? qy[q] : S(0), qT ? qT[q] : S(0)};
        S g[9];
        moments_vjp(M, rho, ux, uy, T, h, g);
#pragma unroll
        for (int i = 0; i < 9; ++i) abar[i * n + q] = g[i];
    }
}

// Initial-field gradient: qbar = sum_i abar_i dF_i/dq at the fields q.
template <typename S>
__global__ void k_feq_vjp(const S* __restrict__ r, const S* __restrict__ ux, const S* __restrict__ uy,
                          const S* __restrict__ T, const S* __restrict__ abar, S* __restrict__ gr,
                          S* __restrict__ gx, S* __restrict__ gy, S* __restrict__ gT, const Model<S> M,
                          long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        S av[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) av[i] = abar[i * n + q];
        S h[4];
        feq_vjp(M, r[q], ux[q], uy[q], T[q], av, h);
        if (gr) gr[q] = h[0];
        if (gx) gx[q] = h[1];
        if (gy) gy[q] = h[2];
        if (gT) gT[q] = h[3];
    }
}
}  // namespace

template <typename S, int TM>
cudaError_t launch_adjoint(const S* f, const S* a, S* abar, const Model<S>& M, const Grid<S>& G,
                           long long level, double* taup, cudaStream_t st) {
    const long long n = (long long)G.nx * G.ny;
    k_adjoint<S, TM><<<blocks_for(n, kThreads), kThreads, 0, st>>>(f, a, abar, M, G, level, taup);
    return cudaGetLastError();
}

template <int TM>
cudaError_t launch_adjoint_tile(const CUtensorMap& tmapA, const CUtensorMap& tmapF, float* abar,
                                const Model<float>& M, const Grid<float>& G, long long level, double* taup,
                                unsigned* status, cudaStream_t st) {
    auto kern = k_adjoint_tile<TM>;
    cudaError_t e = allow_smem<k_adjoint_tile<TM>>(kAdjSmem);
    if (e != cudaSuccess) return e;
    const int tiles_x = (G.nx + kAdjTX - 1) / kAdjTX;
    const int ntiles = tiles_x * ((G.ny + kAdjTY - 1) / kAdjTY);
    const int wave = full_wave<k_adjoint_tile<TM>>(kAdjThreads, kAdjSmem);
    const int grid = ntiles < wave ? ntiles : wave;
    // each step a programmatic dependent of the previous launch on the
    // stream: its CTAs are scheduled while the previous grid drains.  (Tiles
    // claimed at run time, as the forward kernel's double-float mode does,
    // measured slower here: 29.3 -> 32.3 ms for the 1000 adjoint steps of the
    // 2048 x 256 tube; an adjoint tile is short next to the claim's round
    // trip.)
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kAdjThreads);
    lc.dynamicSmemBytes = kAdjSmem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kern, tmapA, tmapF, abar, M, G, level, taup, tiles_x, ntiles, status);
}

cudaError_t launch_adjoint_wrap(float* a, const Grid<float>& G, cudaStream_t st) {
    if (G.kind_lo[S_LEFT] != BC_PERIODIC && G.kind_lo[S_BOTTOM] != BC_PERIODIC) return cudaSuccess;
    k_adjoint_wrap<<<blocks_for((long long)G.nx * G.ny, kThreads), kThreads, 0, st>>>(a, G);
    return cudaGetLastError();
}

void adjoint_tile_boxes(int* ax, int* ay, int* fx, int* fy) {
    *ax = kAdjBoxX;
    *ay = kAdjBoxY;
    *fx = kAdjTX;
    *fy = kAdjTY;
}

// Slots of the tau partials: one per block of the thread-per-node kernel,
// and at least one per CTA of the tile kernel (whose grid never exceeds its
// tile count).
template <typename S>
int adjoint_partials(const Grid<S>& G) {
    const int simple = (int)blocks_for((long long)G.nx * G.ny, kThreads);
    const int tiles = ((G.nx + kAdjTX - 1) / kAdjTX) * ((G.ny + kAdjTY - 1) / kAdjTY);
    return simple > tiles ? simple : tiles;
}

template <typename S, int TM>
cudaError_t launch_moments_vjp(const S* f, const S* qr, const S* qx, const S* qy, const S* qT, S* abar,
                               const Model<S>& M, const Grid<S>& G, cudaStream_t st) {
    unsigned nb = blocks_for((long long)G.nx * G.ny, kThreads);
    if (nb > 65535u * 4u) nb = 65535u * 4u;
    k_moments_vjp<S, TM><<<nb, kThreads, 0, st>>>(f, qr, qx, qy, qT, abar, M, G);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_feq_vjp(const S* r, const S* ux, const S* uy, const S* T, const S* abar, S* gr, S* gx,
                           S* gy, S* gT, const Model<S>& M, long long n, cudaStream_t st) {
    unsigned nb = blocks_for(n, kThreads);
    if (nb > 65535u * 4u) nb = 65535u * 4u;
    k_feq_vjp<S><<<nb, kThreads, 0, st>>>(r, ux, uy, T, abar, gr, gx, gy, gT, M, n);
    return cudaGetLastError();
}

#define LBM_ADJ_INST(S, TM)                                                                             \
    template cudaError_t launch_adjoint<S, TM>(const S*, const S*, S*, const Model<S>&, const Grid<S>&, \
                                               long long, double*, cudaStream_t);                       \
    template cudaError_t launch_moments_vjp<S, TM>(const S*, const S*, const S*, const S*, const S*, S*, \
                                                   const Model<S>&, const Grid<S>&, cudaStream_t);
LBM_ADJ_INST(double, T_PLAIN)
LBM_ADJ_INST(float, T_INT32)
LBM_ADJ_INST(float, T_INT64)
LBM_ADJ_INST(float, T_DF)
LBM_ADJ_INST(float, T_CONS)
#undef LBM_ADJ_INST
template cudaError_t launch_adjoint_tile<T_INT32>(const CUtensorMap&, const CUtensorMap&, float*,
                                                  const Model<float>&, const Grid<float>&, long long, double*,
                                                  unsigned*, cudaStream_t);
template cudaError_t launch_adjoint_tile<T_INT64>(const CUtensorMap&, const CUtensorMap&, float*,
                                                  const Model<float>&, const Grid<float>&, long long, double*,
                                                  unsigned*, cudaStream_t);
template cudaError_t launch_adjoint_tile<T_DF>(const CUtensorMap&, const CUtensorMap&, float*,
                                               const Model<float>&, const Grid<float>&, long long, double*,
                                               unsigned*, cudaStream_t);
template cudaError_t launch_adjoint_tile<T_CONS>(const CUtensorMap&, const CUtensorMap&, float*,
                                                 const Model<float>&, const Grid<float>&, long long, double*,
                                                 unsigned*, cudaStream_t);
template int adjoint_partials<double>(const Grid<double>&);
template int adjoint_partials<float>(const Grid<float>&);
template cudaError_t launch_feq_vjp<double>(const double*, const double*, const double*, const double*,
                                            const double*, double*, double*, double*, double*,
                                            const Model<double>&, long long, cudaStream_t);
template cudaError_t launch_feq_vjp<float>(const float*, const float*, const float*, const float*,
                                           const float*, float*, float*, float*, float*,
                                           const Model<float>&, long long, cudaStream_t);

}  // namespace lbm
