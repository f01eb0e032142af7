// lbm_aux.cu -- initialisation, ghost fill, moments output, FP64 conservation
// totals and interior pack/unpack kernels of liblbm.
#include "lbm_launch.h"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {
constexpr int kThreads = 256;

inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }
}  // namespace

// f = f^eq(rho, u, T) (Eqs. e16-e18) at each interior node.
template <typename S>
__global__ void k_init(S* __restrict__ f, const S* __restrict__ rho, const S* __restrict__ ux,
                       const S* __restrict__ uy, const S* __restrict__ T, const Model<S> M,
                       const Grid<S> G) {
    const long long n = (long long)G.nx * G.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(q / G.nx), ix = (int)(q % G.nx);
        S fe[9];
        equilibrium(M, rho[q], ux[q], uy[q], T[q], fe);
        const size_t c = cell(G, ix, iy);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * (size_t)G.plane + c] = fe[i];
    }
}

template <typename S>
cudaError_t launch_init(S* f, const S* rho, const S* ux, const S* uy, const S* T,
                        const Model<S>& M, const Grid<S>& G, cudaStream_t st) {
    const long long n = (long long)G.nx * G.ny;
    unsigned nb = blocks_for(n, kThreads);
    if (nb > 65535u * 4u) nb = 65535u * 4u;
    k_init<S><<<nb, kThreads, 0, st>>>(f, rho, ux, uy, T, M, G);
    return cudaGetLastError();
}

// Every edge node writes the ghost cells it is responsible for (the same rule
// the step kernel applies to its output level).
template <typename S>
__global__ void k_fill_ghosts(S* __restrict__ f, const Grid<S> G, long long level) {
    const long long total = 2LL * G.nx + 2LL * G.ny;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= total) return;
    int ix, iy;
    if (q < G.nx) {
        ix = (int)q, iy = 0;
    } else if (q < 2LL * G.nx) {
        ix = (int)(q - G.nx), iy = G.ny - 1;
    } else if (q < 2LL * G.nx + G.ny) {
        ix = 0, iy = (int)(q - 2LL * G.nx);
    } else {
        ix = G.nx - 1, iy = (int)(q - 2LL * G.nx - G.ny);
    }
    const size_t c = cell(G, ix, iy);
    S v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = f[i * (size_t)G.plane + c];
    write_ghosts(G, f, ix, iy, v, level);
}

template <typename S>
cudaError_t launch_fill_ghosts(S* f, const Grid<S>& G, long long level, cudaStream_t st) {
    const long long total = 2LL * G.nx + 2LL * G.ny;
    k_fill_ghosts<S><<<blocks_for(total, kThreads), kThreads, 0, st>>>(f, G, level);
    return cudaGetLastError();
}

template <typename S, int TM>
__global__ void k_moments(const S* __restrict__ f, S* __restrict__ rho, S* __restrict__ ux,
                          S* __restrict__ uy, S* __restrict__ T, const Model<S> M, const Grid<S> G,
                          unsigned* status) {
    const long long n = (long long)G.nx * G.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(q / G.nx), ix = (int)(q % G.nx);
        const size_t c = cell(G, ix, iy);
        S v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = f[i * (size_t)G.plane + c];
        S r, u, w, t;
        moments<S, TM>(v, M, r, u, w, t);
        report(status, health(r, u, w, t));
        if (rho) rho[q] = r;
        if (ux) ux[q] = u;
        if (uy) uy[q] = w;
        if (T) T[q] = t;
    }
}

template <typename S, int TM>
cudaError_t launch_moments(const S* f, S* rho, S* ux, S* uy, S* T, const Model<S>& M,
                           const Grid<S>& G, unsigned* status, cudaStream_t st) {
    const long long n = (long long)G.nx * G.ny;
    unsigned nb = blocks_for(n, kThreads);
    if (nb > 65535u * 4u) nb = 65535u * 4u;
    k_moments<S, TM><<<nb, kThreads, 0, st>>>(f, rho, ux, uy, T, M, G, status);
    return cudaGetLastError();
}

// ------------------------------------------------------ conservation totals
// FP64 totals of rho, rho ux, rho uy and E = sum f (v^2 + eta^2) over the
// interior.  Each block reduces a fixed, strided subset of the nodes in a
// fixed tree order; a second single-block pass adds the block partials in a
// fixed order, so the result does not depend on scheduling.
constexpr int kConsBlocks = 1024;

template <typename S>
int conservation_partials(const Grid<S>& G) {
    const long long n = (long long)G.nx * G.ny;
    long long nb = (n + kThreads - 1) / kThreads;
    return (int)(nb < kConsBlocks ? (nb < 1 ? 1 : nb) : kConsBlocks);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_cons_partial(const S* __restrict__ f,
                                                           const Model<double> M,
                                                           const Grid<S> G,
                                                           double* __restrict__ partials) {
    __shared__ double sh[4][kThreads];
    const long long n = (long long)G.nx * G.ny;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(q / G.nx), ix = (int)(q % G.nx);
        const size_t c = cell(G, ix, iy);
        double v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = (double)f[i * (size_t)G.plane + c];
        const double s14 = (v[1] + v[3]) + (v[2] + v[4]);
        const double s58 = (v[5] + v[7]) + (v[6] + v[8]);
        acc[0] += v[0] + s14 + s58;
        acc[1] += M.c1 * (v[3] - v[1]) + M.d * ((v[6] + v[7]) - (v[5] + v[8]));
        acc[2] += M.c1 * (v[4] - v[2]) + M.d * ((v[7] + v[8]) - (v[5] + v[6]));
        acc[3] += M.eta2 * v[0] + M.c1s * s14 + M.c2s * s58;
    }
    block_sum4<kThreads>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) partials[q * gridDim.x + blockIdx.x] = acc[q];
}

__global__ void __launch_bounds__(kThreads) k_cons_final(const double* __restrict__ partials,
                                                         int nparts, double* __restrict__ out) {
    __shared__ double sh[4][kThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nparts; b += kThreads)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += partials[q * nparts + b];
    block_sum4<kThreads>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = acc[q];
}

template <typename S>
cudaError_t launch_conservation(const S* f, const Model<double>& M, const Grid<S>& G,
                                double* partials, double* out, cudaStream_t st) {
    const int nb = conservation_partials(G);
    k_cons_partial<S><<<nb, kThreads, 0, st>>>(f, M, G, partials);
    k_cons_final<<<1, kThreads, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

// ----------------------------------------------------------- pack / unpack
template <typename S>
__global__ void k_pack(const S* __restrict__ f, S* __restrict__ dense, const Grid<S> G, int dir) {
    const long long n = (long long)G.nx * G.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 9 * n;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / n);
        const long long r = q - i * n;
        const int iy = (int)(r / G.nx), ix = (int)(r % G.nx);
        const size_t c = i * (size_t)G.plane + cell(G, ix, iy);
        if (dir == 0)
            dense[q] = f[c];
        else
            const_cast<S*>(f)[c] = dense[q];
    }
}

template <typename S>
cudaError_t launch_pack(const S* f, S* dense, const Grid<S>& G, cudaStream_t st) {
    unsigned nb = blocks_for(9LL * G.nx * G.ny, kThreads);
    if (nb > 65535u * 4u) nb = 65535u * 4u;
    k_pack<S><<<nb, kThreads, 0, st>>>(f, dense, G, 0);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_unpack(S* f, const S* dense, const Grid<S>& G, cudaStream_t st) {
    unsigned nb = blocks_for(9LL * G.nx * G.ny, kThreads);
    if (nb > 65535u * 4u) nb = 65535u * 4u;
    k_pack<S><<<nb, kThreads, 0, st>>>(f, const_cast<S*>(dense), G, 1);
    return cudaGetLastError();
}

#define LBM_INST(S)                                                                          \
    template cudaError_t launch_init<S>(S*, const S*, const S*, const S*, const S*,          \
                                        const Model<S>&, const Grid<S>&, cudaStream_t);      \
    template cudaError_t launch_fill_ghosts<S>(S*, const Grid<S>&, long long, cudaStream_t); \
    template int conservation_partials<S>(const Grid<S>&);                                   \
    template cudaError_t launch_conservation<S>(const S*, const Model<double>&,              \
                                                const Grid<S>&, double*, double*,            \
                                                cudaStream_t);                               \
    template cudaError_t launch_pack<S>(const S*, S*, const Grid<S>&, cudaStream_t);         \
    template cudaError_t launch_unpack<S>(S*, const S*, const Grid<S>&, cudaStream_t);
LBM_INST(double)
LBM_INST(float)
#undef LBM_INST

template cudaError_t launch_moments<double, T_PLAIN>(const double*, double*, double*, double*,
                                                     double*, const Model<double>&,
                                                     const Grid<double>&, unsigned*, cudaStream_t);
template cudaError_t launch_moments<float, T_INT32>(const float*, float*, float*, float*, float*,
                                                    const Model<float>&, const Grid<float>&,
                                                    unsigned*, cudaStream_t);
template cudaError_t launch_moments<float, T_INT64>(const float*, float*, float*, float*, float*,
                                                    const Model<float>&, const Grid<float>&,
                                                    unsigned*, cudaStream_t);
template cudaError_t launch_moments<float, T_DF>(const float*, float*, float*, float*, float*,
                                                 const Model<float>&, const Grid<float>&,
                                                 unsigned*, cudaStream_t);
template cudaError_t launch_moments<float, T_CONS>(const float*, float*, float*, float*, float*,
                                                 const Model<float>&, const Grid<float>&,
                                                 unsigned*, cudaStream_t);

}  // namespace lbm
