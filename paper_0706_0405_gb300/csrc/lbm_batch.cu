// lbm_batch.cu -- many independent problems (each its own grid, constants and
// boundary kinds) advanced by one persistent cooperative launch: every CTA
// walks a static share of the (problem, 256 x 4 tile) list per step, and a
// bounded grid barrier separates the steps.  The per-node arithmetic is the
// vectorised node-group update of the single-grid path (vec_group), so each
// problem's levels are bit-identical to stepping it alone.
#include "lbm_launch.h"

namespace lbm {

namespace {
constexpr int kBatchThreads = 256;
constexpr int kTileW = 256;  // columns per tile (64 threads x 4 nodes)
constexpr int kTileH = 4;    // rows per tile
constexpr long long kBarrierCycles = 4000000000LL;  // ~2 s at 2 GHz, then give up

// Bounded grid-wide barrier for a cooperative launch.  Returns false (and
// sets ST_TIMEOUT) if the barrier did not complete in time.
__device__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == gridDim.x - 1) {
            *count = 0u;
            __threadfence();
            atomicAdd(const_cast<unsigned*>(gen), 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > kBarrierCycles) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <typename S>
__device__ __forceinline__ void copy_words(S* dst, const S* src, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

template <int TM>
__global__ void __launch_bounds__(kBatchThreads)
    k_batch(const BatchProb* __restrict__ probs, const int4* __restrict__ tiles, int ntiles, int nsteps,
            long long* level_ptr, unsigned* bar_count, unsigned* bar_gen, unsigned* status) {
    __shared__ Model<float> sM;
    __shared__ Grid<float> sG;
    const long long level0 = *(volatile long long*)level_ptr;
    unsigned bits = 0;
    const int r = threadIdx.x / (kTileW / 4);        // row inside the tile
    const int g4 = (threadIdx.x % (kTileW / 4)) * 4;  // first column of my group inside the tile
    for (int s = 0; s < nsteps; ++s) {
        const long long level = level0 + s;
        const int par = (int)(level & 1);
        if (*(volatile unsigned*)status & ST_TIMEOUT) return;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int4 T = tiles[t];
            const BatchProb& P = probs[T.x];
            __syncthreads();
            copy_words(reinterpret_cast<float*>(&sM), reinterpret_cast<const float*>(&P.M),
                       (int)(sizeof(Model<float>) / sizeof(float)));
            copy_words(reinterpret_cast<int*>(&sG), reinterpret_cast<const int*>(&P.G),
                       (int)(sizeof(Grid<float>) / sizeof(int)));
            __syncthreads();
            const int ix0 = T.y + g4, iy = T.z + r;
            if (ix0 < sG.nx && iy < sG.ny)
                bits |= vec_group<4, TM, true>(P.f[par], P.f[par ^ 1], sM, sG, ix0, iy, level);
        }
        if (!grid_barrier(bar_count, bar_gen, status)) return;
    }
    report(status, bits);
    if (blockIdx.x == 0 && threadIdx.x == 0) *level_ptr = level0 + nsteps;
}
}  // namespace

int batch_tile_dims(int* w, int* h) {
    *w = kTileW;
    *h = kTileH;
    return kBatchThreads;
}

template <int TM>
cudaError_t launch_batch(const BatchProb* probs, const int4* tiles, int ntiles, int nsteps, long long* level,
                         unsigned* bar_count, unsigned* bar_gen, unsigned* status, int grid, cudaStream_t st) {
    auto kern = k_batch<TM>;
    void* args[] = {(void*)&probs, (void*)&tiles, (void*)&ntiles, (void*)&nsteps,
                    (void*)&level,  (void*)&bar_count, (void*)&bar_gen, (void*)&status};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

template <int TM>
int batch_max_grid() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<TM>, kBatchThreads, 0);
    return sms * (per_sm > 0 ? per_sm : 1);
}

template cudaError_t launch_batch<T_INT32>(const BatchProb*, const int4*, int, int, long long*, unsigned*,
                                           unsigned*, unsigned*, int, cudaStream_t);
template cudaError_t launch_batch<T_INT64>(const BatchProb*, const int4*, int, int, long long*, unsigned*,
                                           unsigned*, unsigned*, int, cudaStream_t);
template cudaError_t launch_batch<T_DF>(const BatchProb*, const int4*, int, int, long long*, unsigned*,
                                        unsigned*, unsigned*, int, cudaStream_t);
template int batch_max_grid<T_INT32>();
template int batch_max_grid<T_INT64>();
template int batch_max_grid<T_DF>();

}  // namespace lbm
