// lbm_batch.cu -- many independent problems (each its own grid, constants and
// boundary kinds) advanced by one persistent cooperative launch: every CTA
// walks a contiguous share of the (problem, 64 x 4 tile) list per step, and a
// bounded grid barrier separates the steps.  Each tile and its halo (72 x 6
// x 9 floats) are loaded into shared memory by all threads with 16-byte
// reads through L2 (data of the previous step written by other CTAs), then
// every thread updates one node with the same per-node arithmetic as the
// single-grid kernels, so each problem's levels are bit-identical to stepping
// it alone.
#include "lbm_launch.h"

namespace lbm {

namespace {
constexpr int kBatchThreads = 256;
constexpr int kTileW = 64;  // columns per tile (one node per thread)
constexpr int kTileH = 4;   // rows per tile
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

constexpr int kBoxW = kTileW + 8;  // 4 extra columns each side keep 16-byte alignment
constexpr int kBoxH = kTileH + 2;
constexpr int kBoxPlane = kBoxW * kBoxH;

template <int TM>
__global__ void __launch_bounds__(kBatchThreads)
    k_batch(const BatchProb* __restrict__ probs, const int4* __restrict__ tiles, int ntiles, int nsteps,
            long long* level_ptr, unsigned* bar_count, unsigned* bar_gen, unsigned* status) {
    __shared__ Model<float> sM;
    __shared__ Grid<float> sG;
    __shared__ __align__(16) float box[9 * kBoxPlane];
    const long long level0 = *(volatile long long*)level_ptr;
    unsigned bits = 0;
    const int r = threadIdx.x / kTileW, cx = threadIdx.x % kTileW;
    // a contiguous run of tiles per CTA: consecutive tiles mostly share a
    // problem, so its constants are copied to shared memory rarely
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per, t1 = min(ntiles, t0 + per);
    constexpr int kVecs = 9 * kBoxH * (kBoxW / 4);  // float4 loads per box
    for (int s = 0; s < nsteps; ++s) {
        const long long level = level0 + s;
        const int par = (int)(level & 1);
        if (*(volatile unsigned*)status & ST_TIMEOUT) return;
        int cur = -1;
        for (int t = t0; t < t1; ++t) {
            const int4 T = tiles[t];
            const BatchProb& P = probs[T.x];
            __syncthreads();  // previous tile's box (and constants) no longer read
            if (T.x != cur) {
                copy_words(reinterpret_cast<float*>(&sM), reinterpret_cast<const float*>(&P.M),
                           (int)(sizeof(Model<float>) / sizeof(float)));
                copy_words(reinterpret_cast<int*>(&sG), reinterpret_cast<const int*>(&P.G),
                           (int)(sizeof(Grid<float>) / sizeof(int)));
                cur = T.x;
            }
            // box: array rows T.z .. T.z + kBoxH - 1 (interior rows T.z - 1 ..),
            // array columns T.y .. T.y + kBoxW - 1 (interior columns T.y - 4 ..);
            // whole float4 groups inside the row pitch only (the columns any
            // node reads always are), read through L2
            const float* fin = P.f[par];
            const int pitch = P.G.pitch, rows = P.G.ny + 2;
            const size_t pl = (size_t)P.G.plane;
            for (int v = threadIdx.x; v < kVecs; v += kBatchThreads) {
                const int i = v / (kBoxH * (kBoxW / 4));
                const int rem = v % (kBoxH * (kBoxW / 4));
                const int yy = rem / (kBoxW / 4), xx = (rem % (kBoxW / 4)) * 4;
                const int ay = T.z + yy, ax = T.y + xx;
                if (ay < rows && ax + 4 <= pitch) {
                    const float4 q = __ldcg(reinterpret_cast<const float4*>(fin + i * pl + (size_t)ay * pitch + ax));
                    *reinterpret_cast<float4*>(&box[i * kBoxPlane + yy * kBoxW + xx]) = q;
                }
            }
            __syncthreads();
            const int ix = T.y + cx, iy = T.z + r;
            if (ix < sG.nx && iy < sG.ny) {
                const float* b = box + (r + 1) * kBoxW + (cx + 4);
                float f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = b[i * kBoxPlane];
                float rho, ux, uy, Tt;
                moments<float, TM>(f, sM, rho, ux, uy, Tt);
                bits |= health(rho, ux, uy, Tt);
                float ofe[9], o[9];
                relaxation<float, TM>(sM, f, rho, ux, uy, Tt, ofe);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float* bp = b + i * kBoxPlane;
                    o[i] = update(sM, i, ofe[i], f[i], bp[1], bp[-1], bp[kBoxW], bp[-kBoxW]);
                }
                float* fout = P.f[par ^ 1];
                const size_t c = cell(sG, ix, iy);
#pragma unroll
                for (int i = 0; i < 9; ++i) fout[i * pl + c] = o[i];
                if (ix == 0 || iy == 0 || ix == sG.nx - 1 || iy == sG.ny - 1)
                    write_ghosts(sG, fout, ix, iy, o, level + 1);
            }
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
template cudaError_t launch_batch<T_CONS>(const BatchProb*, const int4*, int, int, long long*, unsigned*,
                                          unsigned*, unsigned*, int, cudaStream_t);
template int batch_max_grid<T_INT32>();
template int batch_max_grid<T_INT64>();
template int batch_max_grid<T_DF>();
template int batch_max_grid<T_CONS>();

}  // namespace lbm
