// lbm_noalloc.cu -- lbm_conservation_noalloc: the FP64 conservation totals of
// a distribution the caller already holds, computed without allocating any
// memory.
//
// Who needs it: callers that cannot make CUDA allocations at the point where
// they want the totals, e.g. a process whose device memory is entirely
// committed to a pre-allocated pool or a framework's caching allocator (a
// cudaMalloc outside that pool fails or fragments it), a latency-critical
// loop in which cudaMalloc / cudaFree could synchronise the device and stall
// it, or a host that enforces a fixed device-memory budget.  lbm_conservation
// needs a context, and a context allocates its buffers; this entry point needs
// neither.
//
// Scratch: the per-tile partial sums and the result live in the file-scope
// array g_scratch below (kScratchDoubles doubles, 64 KiB + 32 B).  Every GPU
// that loads the library holds this array until the process exits.  All calls
// share it and it keeps the last call's contents; each call writes every
// partial it later reads and the final result, so nothing has to start at
// zero.  Calls that overlap on the GPU (on different streams, or from
// different host threads without ordering) race on the array and may return
// wrong totals: order them.
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_reduce.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 16;
constexpr long long kTile = (long long)kThreads * kNodesPerThread;  // nodes per CTA
constexpr int kMaxTiles = 2048;                                     // partial quadruples held
constexpr long long kMaxNodes = kTile * kMaxTiles;                  // 8 388 608 nodes
constexpr int kScratchDoubles = 4 * kMaxTiles + 4;                  // partials + result

__device__ __align__(256) double g_scratch[kScratchDoubles];

// Device addresses of g_scratch, one per CUDA context that has called in.
// The symbol's name is only a host-side stand-in: its device address belongs
// to the module as loaded in one context, so it is looked up (with that
// context current) the first time a context calls, and kept under the
// context's unique ID, which the driver never hands out twice.  A caller on a
// non-primary context, or on a new primary context after cudaDeviceReset,
// therefore gets an address of its own context.  Without the driver's
// context queries the address is looked up on every call.
struct ScratchAddr {
    unsigned long long ctx_id;
    double* ptr;
};
std::vector<ScratchAddr> g_scratch_addrs;
std::mutex g_setup_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

template <typename Fn>
Fn driver_fn(const char* name, int version) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return reinterpret_cast<Fn>(p);
}

// The current context's unique ID, or 0 if it cannot be had.
unsigned long long current_context_id() {
    static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 4000);
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// &g_scratch in the current context (nullptr on failure).  Call with the
// caller's device current and the runtime initialised on it.
double* scratch_address() {
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (id != 0)
        for (const ScratchAddr& a : g_scratch_addrs)
            if (a.ctx_id == id) return a.ptr;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (id != 0) g_scratch_addrs.push_back({id, static_cast<double*>(p)});
    return static_cast<double*>(p);
}

// Partial totals of one tile of kTile nodes of a dense 9 x n distribution
// (rho, rho ux, rho uy, E = sum f (v^2 + eta^2), the sums of Eqs. e4, e5, e7
// of the paper), written to scratch[q * ntiles + tile].
template <typename S>
__global__ void __launch_bounds__(kThreads)
    k_totals_tiles(const S* __restrict__ f, long long n, double c1, double d, double c1s, double c2s,
                   double eta2, double* __restrict__ scratch) {
    __shared__ double sh[4][kThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * kTile;
    for (int k = 0; k < kNodesPerThread; ++k) {
        const long long q = base + (long long)k * kThreads + threadIdx.x;
        if (q >= n) break;
        double v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = (double)f[(long long)i * n + q];
        const double s14 = (v[1] + v[3]) + (v[2] + v[4]);
        const double s58 = (v[5] + v[7]) + (v[6] + v[8]);
        acc[0] += v[0] + s14 + s58;
        acc[1] += c1 * (v[3] - v[1]) + d * ((v[6] + v[7]) - (v[5] + v[8]));
        acc[2] += c1 * (v[4] - v[2]) + d * ((v[7] + v[8]) - (v[5] + v[6]));
        acc[3] += eta2 * v[0] + c1s * s14 + c2s * s58;
    }
    lbm::block_sum4<kThreads>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) scratch[q * gridDim.x + blockIdx.x] = acc[q];
}

// Sum the ntiles partials of each quantity in a fixed order into
// scratch[4 * kMaxTiles + q].
__global__ void __launch_bounds__(kThreads) k_totals_final(double* __restrict__ scratch, int ntiles) {
    __shared__ double sh[4][kThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < ntiles; b += kThreads)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += scratch[q * ntiles + b];
    lbm::block_sum4<kThreads>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) scratch[4 * kMaxTiles + q] = acc[q];
}

}  // namespace

extern "C" lbm_status lbm_conservation_noalloc(const void* f, int nx, int ny, lbm_precision prec,
                                               const lbm_dvm* dvm, double out[4], void* stream) {
    if (!f || !dvm || !out) return LBM_E_INVAL;
    if (nx < 1 || ny < 1) return LBM_E_INVAL;
    const long long n = (long long)nx * (long long)ny;
    if (n > kMaxNodes) return LBM_E_INVAL;  // more tiles than the static scratch holds
    if (prec < LBM_FP64 || prec > LBM_FP32_CONS) return LBM_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    double* scratch = scratch_address();
    if (!scratch) return LBM_E_CUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ntiles = (int)((n + kTile - 1) / kTile);
    const double d = dvm->c2 / std::sqrt(2.0);
    if (prec == LBM_FP64)
        k_totals_tiles<double><<<ntiles, kThreads, 0, st>>>(static_cast<const double*>(f), n, dvm->c1, d,
                                                            dvm->c1 * dvm->c1, dvm->c2 * dvm->c2,
                                                            dvm->eta0 * dvm->eta0, scratch);
    else
        k_totals_tiles<float><<<ntiles, kThreads, 0, st>>>(static_cast<const float*>(f), n, dvm->c1, d,
                                                           dvm->c1 * dvm->c1, dvm->c2 * dvm->c2,
                                                           dvm->eta0 * dvm->eta0, scratch);
    k_totals_final<<<1, kThreads, 0, st>>>(scratch, ntiles);
    if (cudaGetLastError() != cudaSuccess) return LBM_E_CUDA;
    if (cudaMemcpyAsync(out, scratch + 4 * kMaxTiles, 4 * sizeof(double), cudaMemcpyDefault, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    return LBM_OK;
}
