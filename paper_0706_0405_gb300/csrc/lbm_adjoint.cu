// lbm_adjoint.cu -- the hand-written adjoint of the fused step: the transpose
// of the linearised update of Eq. (SEC-VON-11) (transposed five-point star,
// ghost links through the boundary rule, transposed collision Jacobian), the
// tau derivative, and the vector-Jacobian products of the equilibrium
// (Eqs. e16-e18) and of the moments (Eqs. e4, e5, e7).
#include "lbm_launch.h"
#include "lbm_linear.cuh"

namespace lbm {

namespace {
constexpr int kThreads = 256;

inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

template <typename S>
__device__ __forceinline__ int kind_at(const Grid<S>& G, int side, int along_index, long long level) {
    return side_part(G, side, along_index, level) ? G.kind_hi[side] : G.kind_lo[side];
}

// One adjoint step from level n + 1 back to level n (gather form over the
// transposed star).  a: adjoint of level n + 1, abar: adjoint of level n
// (interior of the padded layout; ghost cells are never read or written).
// taup[block] += sum over the block's nodes of sum_i a_i (f^eq_i - f_i)
// (per node in the storage precision, across nodes in FP64; the tau
// derivative is -(dt / tau^2) times the total).
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
        S fv[9], av[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fv[i] = f[i * pl + c];
            av[i] = a[i * pl + c];
        }
        S rho, ux, uy, T;
        moments<S, TM>(fv, M, rho, ux, uy, T);
        S fe[9];
        equilibrium(M, rho, ux, uy, T, fe);
        // sum_i a_i (f^eq_i - f_i) in the storage precision per node; the
        // sum over nodes is FP64
        S tn = S(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) tn += av[i] * (fe[i] - fv[i]);
        tsum = tn;
        S h[4], g[9];
        feq_vjp(M, rho, ux, uy, T, av, h);
        moments_vjp(M, rho, ux, uy, T, h, g);
        // neighbour sources of the transposed star, with periodic wrap
        const bool perx = G.kind_lo[S_LEFT] == BC_PERIODIC;
        const bool pery = G.kind_lo[S_BOTTOM] == BC_PERIODIC;
        const int xl = ix > 0 ? ix - 1 : (perx ? G.nx - 1 : -1);
        const int xr = ix < G.nx - 1 ? ix + 1 : (perx ? 0 : -1);
        const int yd = iy > 0 ? iy - 1 : (pery ? G.ny - 1 : -1);
        const int yu = iy < G.ny - 1 ? iy + 1 : (pery ? 0 : -1);
        const int kl = ix == 0 ? kind_at(G, S_LEFT, iy, level) : -1;
        const int kr = ix == G.nx - 1 ? kind_at(G, S_RIGHT, iy, level) : -1;
        const int kb = iy == 0 ? kind_at(G, S_BOTTOM, ix, level) : -1;
        const int kt = iy == G.ny - 1 ? kind_at(G, S_TOP, ix, level) : -1;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            S o = M.w[j][0] * av[j] + M.omega * g[j];
            if (xl >= 0) o += M.w[j][1] * a[j * pl + cell(G, xl, iy)];  // node left of me reads me as E
            if (xr >= 0) o += M.w[j][2] * a[j * pl + cell(G, xr, iy)];  // node right of me reads me as W
            if (yd >= 0) o += M.w[j][3] * a[j * pl + cell(G, ix, yd)];  // node below reads me as N
            if (yu >= 0) o += M.w[j][4] * a[j * pl + cell(G, ix, yu)];  // node above reads me as S
            // ghost links: my own ghost on a non-periodic side is made from me
            if (kl == BC_OUTFLOW) o += M.w[j][2] * av[j];
            if (kl == BC_REFLECT) o += M.w[mirror_x(j)][2] * av[mirror_x(j)];
            if (kr == BC_OUTFLOW) o += M.w[j][1] * av[j];
            if (kr == BC_REFLECT) o += M.w[mirror_x(j)][1] * av[mirror_x(j)];
            if (kb == BC_OUTFLOW) o += M.w[j][4] * av[j];
            if (kb == BC_REFLECT) o += M.w[mirror_y(j)][4] * av[mirror_y(j)];
            if (kt == BC_OUTFLOW) o += M.w[j][3] * av[j];
            if (kt == BC_REFLECT) o += M.w[mirror_y(j)][3] * av[mirror_y(j)];
            abar[j * pl + c] = o;
        }
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

template <typename S>
int adjoint_partials(const Grid<S>& G) {
    return (int)blocks_for((long long)G.nx * G.ny, kThreads);
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
template int adjoint_partials<double>(const Grid<double>&);
template int adjoint_partials<float>(const Grid<float>&);
template cudaError_t launch_feq_vjp<double>(const double*, const double*, const double*, const double*,
                                            const double*, double*, double*, double*, double*,
                                            const Model<double>&, long long, cudaStream_t);
template cudaError_t launch_feq_vjp<float>(const float*, const float*, const float*, const float*,
                                           const float*, float*, float*, float*, float*,
                                           const Model<float>&, long long, cudaStream_t);

}  // namespace lbm
