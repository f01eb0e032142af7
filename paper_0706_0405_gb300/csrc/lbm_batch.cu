// lbm_batch.cu -- many independent problems (each its own grid, constants and
// boundary kinds) advanced by one persistent cooperative launch: every CTA
// walks a contiguous share of the (problem, 64 x 4 tile) list per step, and a
// bounded grid barrier separates the steps.  Each tile and its halo (72 x 6
// x 9 floats) arrive in shared memory by one tiled tensor copy through the
// problem's own tensor map, double-buffered so that the next tile of the
// CTA's share is in flight while the current one is computed; every thread
// then updates one node with the same per-node arithmetic as the single-grid
// kernels, so each problem's levels are bit-identical to stepping it alone.
#include "lbm_launch.h"
#include "lbm_ptx.cuh"

namespace lbm {

namespace {
constexpr int kTileW = 64;  // columns per tile
constexpr int kTileH = 4;   // rows per tile
// threads per CTA for NPT x-adjacent nodes per thread (1 or 2)
template <int NPT>
constexpr int batch_threads() {
    return kTileW / NPT * kTileH;
}
constexpr long long kBarrierCycles = 4000000000LL;  // ~2 s at 2 GHz, then give up
constexpr uint32_t kBatchWaitLimit = 1u << 22;       // mbarrier probes before a wait gives up

// Bounded grid-wide barrier for a cooperative launch.  Returns false (and
// sets ST_TIMEOUT) if the barrier did not complete in time.  The stores of
// the step are ordered before the async-proxy reads (tensor copies) of the
// next step on both sides: every thread fences after its stores, and the
// thread that issues the copies fences after the barrier.
__device__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned* status) {
    __shared__ int ok;
    fence_proxy_async_global();
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
        fence_proxy_async_global();
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
constexpr int kBoxFloats = 9 * kBoxPlane;
constexpr int kStageFloats = (kBoxFloats + 31) / 32 * 32;  // stages on 128-byte boundaries
constexpr size_t kBatchSmem = 128 + sizeof(float) * 2 * kStageFloats + 2 * sizeof(uint64_t);

template <int TM, int NPT>
__global__ void __launch_bounds__(batch_threads<NPT>())
    k_batch(const BatchProb* __restrict__ probs, const int4* __restrict__ tiles, int ntiles, int nsteps,
            long long* level_ptr, unsigned* bar_count, unsigned* bar_gen, unsigned* status) {
    __shared__ Model<float> sM;
    __shared__ Grid<float> sG;
    __shared__ int abort_flag;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    float* box0 = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(float) * 2 * kStageFloats);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    const long long level0 = *(volatile long long*)level_ptr;
    unsigned bits = 0;
    constexpr int kLanesX = kTileW / NPT;  // threads along a tile row
    const int r = tid / kLanesX, cx = tid % kLanesX;
    // a contiguous run of tiles per CTA: consecutive tiles mostly share a
    // problem, so its constants are copied to shared memory rarely
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per, t1 = min(ntiles, t0 + per);
    // running index k of this CTA's tiles over all steps: stage k & 1,
    // phase parity (k >> 1) & 1
    auto issue = [&](int t, int k, int par) {
        const int4 T = tiles[t];
        mbar_arrive_expect_tx(&bar[k & 1], (uint32_t)(sizeof(float) * kBoxFloats));
        // array column T.y (interior column T.y - 4), array row T.z (interior row T.z - 1)
        tma_load_3d(box0 + (k & 1) * kStageFloats, &probs[T.x].tm[par], T.y, T.z, 0, &bar[k & 1]);
    };
    auto wait = [&](int k) { return mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), kBatchWaitLimit); };
    int k = 0, issued = -1, waited = -1;
    for (int s = 0; s < nsteps; ++s) {
        const long long level = level0 + s;
        const int par = (int)(level & 1);
        if (*(volatile unsigned*)status & ST_TIMEOUT) return;
        if (t0 < t1) {
            if (tid == 0) issue(t0, k, par);
            issued = k;
        }
        int cur = -1;
        for (int t = t0; t < t1; ++t, ++k) {
            // one thread waits for tile k; the barrier also says every thread
            // is done with tile k - 1 (its box and the problem constants)
            if (tid == 0 && !wait(k)) abort_flag = 1;
            __syncthreads();
            if (abort_flag) {
                for (int j = waited + 1; j <= issued; ++j) wait(j);
                if (tid == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
            waited = k;
            if (t + 1 < t1) {
                if (tid == 0) issue(t + 1, k + 1, par);
                issued = k + 1;
            }
            const int4 T = tiles[t];
            const BatchProb& P = probs[T.x];
            if (T.x != cur) {
                copy_words(reinterpret_cast<float*>(&sM), reinterpret_cast<const float*>(&P.M),
                           (int)(sizeof(Model<float>) / sizeof(float)));
                copy_words(reinterpret_cast<int*>(&sG), reinterpret_cast<const int*>(&P.G),
                           (int)(sizeof(Grid<float>) / sizeof(int)));
                cur = T.x;
                __syncthreads();
            }
            if constexpr (NPT == 1) {
                const int ix = T.y + cx, iy = T.z + r;
                if (ix < sG.nx && iy < sG.ny) {
                    const float* b = box0 + (k & 1) * kStageFloats + (r + 1) * kBoxW + (cx + 4);
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
                    const size_t pl = (size_t)sG.plane;
                    const size_t c = cell(sG, ix, iy);
#pragma unroll
                    for (int i = 0; i < 9; ++i) fout[i * pl + c] = o[i];
                    if (ix == 0 || iy == 0 || ix == sG.nx - 1 || iy == sG.ny - 1)
                        write_ghosts(sG, fout, ix, iy, o, level + 1);
                }
            } else {  // two x-adjacent nodes per thread, 8-byte shared loads and stores
                const int ix0 = T.y + 2 * cx, iy = T.z + r;
                if (ix0 < sG.nx && iy < sG.ny) {
                    const int nvalid = min(2, sG.nx - ix0);
                    const float* b = box0 + (k & 1) * kStageFloats + (r + 1) * kBoxW + (2 * cx + 4);
                    float2 C[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) C[i] = *reinterpret_cast<const float2*>(b + i * kBoxPlane);
                    float acc[9][2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        float f[9];
#pragma unroll
                        for (int i = 0; i < 9; ++i) f[i] = j ? C[i].y : C[i].x;
                        float rho, ux, uy, Tt;
                        moments<float, TM>(f, sM, rho, ux, uy, Tt);
                        if (j < nvalid) bits |= health(rho, ux, uy, Tt);
                        float ofe[9];
                        relaxation<float, TM>(sM, f, rho, ux, uy, Tt, ofe);
#pragma unroll
                        for (int i = 0; i < 9; ++i) acc[i][j] = ofe[i];
                    }
                    float* fout = P.f[par ^ 1];
                    const size_t pl = (size_t)sG.plane;
                    float* out = fout + cell(sG, ix0, iy);  // 8-byte aligned: ix0 + PADX is even
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const float* bp = b + i * kBoxPlane;
                        const float2 Nn = *reinterpret_cast<const float2*>(bp + kBoxW);
                        const float2 Ss = *reinterpret_cast<const float2*>(bp - kBoxW);
                        const float Wv = bp[-1], Ev = bp[2];
                        float2 o;
                        o.x = update(sM, i, acc[i][0], C[i].x, C[i].y, Wv, Nn.x, Ss.x);
                        o.y = update(sM, i, acc[i][1], C[i].y, Ev, C[i].x, Nn.y, Ss.y);
                        if (nvalid == 2)
                            *reinterpret_cast<float2*>(out + i * pl) = o;
                        else
                            out[i * pl] = o.x;
                    }
                    const bool edge_row = iy == 0 || iy == sG.ny - 1;
                    if (edge_row || ix0 == 0 || ix0 + nvalid == sG.nx) {
                        for (int j = 0; j < nvalid; ++j) {
                            const int ix = ix0 + j;
                            if (!(edge_row || ix == 0 || ix == sG.nx - 1)) continue;
                            float v[9];
#pragma unroll
                            for (int i = 0; i < 9; ++i) v[i] = out[i * pl + j];
                            write_ghosts(sG, fout, ix, iy, v, level + 1);
                        }
                    }
                }
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
    return batch_threads<1>();
}

void batch_box_dims(int* bx, int* by) {
    *bx = kBoxW;
    *by = kBoxH;
}

template <int TM, int NPT>
cudaError_t launch_batch_v(const BatchProb* probs, const int4* tiles, int ntiles, int nsteps, long long* level,
                           unsigned* bar_count, unsigned* bar_gen, unsigned* status, int grid, cudaStream_t st) {
    auto kern = k_batch<TM, NPT>;
    cudaError_t e = allow_smem<k_batch<TM, NPT>>(kBatchSmem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&probs, (void*)&tiles, (void*)&ntiles, (void*)&nsteps,
                    (void*)&level,  (void*)&bar_count, (void*)&bar_gen, (void*)&status};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(batch_threads<NPT>());
    cfg.dynamicSmemBytes = kBatchSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

template <int TM>
cudaError_t launch_batch(const BatchProb* probs, const int4* tiles, int ntiles, int nsteps, long long* level,
                         unsigned* bar_count, unsigned* bar_gen, unsigned* status, int grid, int npt,
                         cudaStream_t st) {
    if (npt == 2)
        return launch_batch_v<TM, 2>(probs, tiles, ntiles, nsteps, level, bar_count, bar_gen, status, grid, st);
    return launch_batch_v<TM, 1>(probs, tiles, ntiles, nsteps, level, bar_count, bar_gen, status, grid, st);
}

template <int TM, int NPT>
int batch_max_grid_v() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    allow_smem<k_batch<TM, NPT>>(kBatchSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<TM, NPT>, batch_threads<NPT>(), kBatchSmem);
    return sms * (per_sm > 0 ? per_sm : 1);
}

template <int TM>
int batch_max_grid(int npt) {
    return npt == 2 ? batch_max_grid_v<TM, 2>() : batch_max_grid_v<TM, 1>();
}

#define LBM_BATCH_INST(TM)                                                                                  \
    template cudaError_t launch_batch<TM>(const BatchProb*, const int4*, int, int, long long*, unsigned*,  \
                                          unsigned*, unsigned*, int, int, cudaStream_t);                   \
    template int batch_max_grid<TM>(int);
LBM_BATCH_INST(T_INT32)
LBM_BATCH_INST(T_INT64)
LBM_BATCH_INST(T_DF)
LBM_BATCH_INST(T_CONS)
#undef LBM_BATCH_INST

}  // namespace lbm
