// lbm_batch.cu -- many independent problems (each its own grid, constants and
// boundary kinds) advanced by one persistent cooperative launch: every CTA
// walks its share of the (problem, 64 x 4 tile) list per step, and a CTA
// starts a step once the CTAs owning the tiles next to its own have finished
// the previous one (bounded waits; a grid barrier where the neighbour lists
// would be too long).  Each tile and its halo (72 x 6 x 9 floats, or the
// 72 x 4 x 9 interior rows of a problem that wraps in y inside one tile row)
// arrive in shared memory by one tiled tensor copy through the problem's own
// tensor map, double-buffered so that the next tile of the CTA's share is in
// flight while the current one is computed; every thread then updates one or
// two nodes with the same per-node arithmetic as the single-grid kernels, so
// each problem's levels are bit-identical to stepping it alone.
#include <cstddef>

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
// SM cycles an inter-CTA wait (grid barrier, neighbour wait) lasts before it
// gives up (batch_set_wait_cycles)
__device__ long long g_wait_cycles = kBarrierCycles;
constexpr uint32_t kBatchWaitLimit = 1u << 22;       // mbarrier probes before a wait gives up

// Bounded grid-wide barrier for a cooperative launch.  Returns false (and
// sets ST_TIMEOUT) if the barrier did not complete in time or another CTA
// has given up (ST_TIMEOUT already set); the decision is the CTA's, taken
// by one thread and passed on by the CTA barrier, so all its threads leave
// together.  The stores of
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
                if (clock64() - t0 > g_wait_cycles || (*(volatile unsigned*)status & ST_TIMEOUT)) {
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

// Point-to-point step ordering between CTAs.  After its last tile of a
// step, a CTA publishes the step count it has completed (a value that only
// grows over the batch's life: the epoch of the launch plus the steps done);
// before a step it waits until every CTA owning a tile next to one of its
// own (the host's neighbour list, periodic partners included) has completed
// the previous step.  That orders both the reads of the halo written by a
// neighbour and the overwriting of the level a neighbour was still reading,
// without making every CTA wait for the slowest one.  Same fences as the
// grid barrier; the wait is bounded, and gives up at once once another CTA
// has given up (ST_TIMEOUT set), the CTA's threads leaving together.
__device__ void publish_step(unsigned long long* done, unsigned long long value) {
    fence_proxy_async_global();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(done + blockIdx.x, value);
    }
}

__device__ bool wait_neighbours(const int* __restrict__ nbr, const unsigned long long* done,
                                unsigned long long target, unsigned* status) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = (*(volatile unsigned*)status & ST_TIMEOUT) ? 0 : 1;
        const long long t0 = clock64();
        for (int j = 0; j < kBatchMaxNbr && ok; ++j) {
            const int n = nbr[j];
            if (n < 0) break;
            while (*(volatile const unsigned long long*)(done + n) < target) {
                if (clock64() - t0 > g_wait_cycles || (*(volatile unsigned*)status & ST_TIMEOUT)) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        fence_proxy_async_global();
    }
    __syncthreads();
    return ok != 0;
}

// A problem whose whole height fits in one tile row and whose bottom and
// top sides are periodic: its tiles hold every row of the level, so the
// wrapped y neighbours come from the box itself and the level's y ghost rows
// need not be stored between the steps of a launch.
__host__ __device__ __forceinline__ bool wraps_in_tile(const Grid<float>& G, int tile_h) {
    return G.ny <= tile_h && G.kind_lo[S_BOTTOM] == BC_PERIODIC && G.kind_hi[S_BOTTOM] == BC_PERIODIC &&
           G.kind_lo[S_TOP] == BC_PERIODIC && G.kind_hi[S_TOP] == BC_PERIODIC;
}

// The ghost cells of level `level` that edge node (ix, iy) writes (as
// write_ghosts), but on the left and right sides only.
__device__ __forceinline__ void write_ghosts_x(const Grid<float>& G, float* __restrict__ f, int ix, int iy,
                                               const float (&v)[9], long long level) {
    const size_t pl = (size_t)G.plane;
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

template <typename S>
__device__ __forceinline__ void copy_words(S* dst, const S* src, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

#ifndef LBM_BATCH_STRIDED
#define LBM_BATCH_STRIDED 0
#endif
constexpr bool kBatchStrided = LBM_BATCH_STRIDED != 0;
constexpr int kBoxW = kTileW + 8;  // 4 extra columns each side keep 16-byte alignment
constexpr int kBoxH = kTileH + 2;
// The box in shared memory is [row][population][column], like the level.
constexpr int kBoxPop = kBoxW, kBoxRow = 9 * kBoxW;  // population and row strides
constexpr int kBoxFloats = kBoxH * kBoxRow;
constexpr int kStageFloats = (kBoxFloats + 31) / 32 * 32;  // stages on 128-byte boundaries
constexpr size_t kBatchSmem = 128 + sizeof(float) * 2 * kStageFloats + 2 * sizeof(uint64_t);

// A problem's constants (its Model and Grid, contiguous in BatchProb) travel
// to shared memory as one bulk copy beside each box that starts a run of the
// problem's tiles in a stage: kConstBytes from offset kConstOff of the record.
constexpr size_t kConstOff = offsetof(BatchProb, M);
constexpr size_t kGridInConst = offsetof(BatchProb, G) - kConstOff;
constexpr size_t kConstBytes = (kGridInConst + sizeof(Grid<float>) + 15) / 16 * 16;
static_assert(kConstOff % 16 == 0, "bulk copies start on 16-byte boundaries");
static_assert(kConstOff + kConstBytes <= sizeof(BatchProb), "the copy stays inside the record");

// CTAs per SM the register allocation must allow: 6 of 128 threads (at most
// 80 registers a thread), 4 of 256 (64)
template <int NPT>
constexpr int batch_min_blocks() {
    return NPT == 2 ? 6 : 4;
}

template <int TM, int NPT>
__global__ void __launch_bounds__(batch_threads<NPT>(), batch_min_blocks<NPT>())
    k_batch(const BatchProb* __restrict__ probs, const int4* __restrict__ tiles, int ntiles, int nsteps,
            long long* level_ptr, unsigned* bar_count, unsigned* bar_gen, unsigned* status,
            const int* __restrict__ nbr, unsigned long long* done, unsigned long long* epoch_ptr) {
    // each stage's problem constants (Model, then Grid at kGridInConst)
    __shared__ __align__(16) unsigned char sConst[2][kConstBytes];
    __shared__ int const_of[2];  // problem whose constants a stage holds (thread 0)
    __shared__ int abort_flag;
    __shared__ int4 stage_T[2];  // the tile entry of the box in each stage
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
        const_of[0] = const_of[1] = -1;
    }
    __syncthreads();
    const long long level0 = *(volatile long long*)level_ptr;
    const unsigned long long epoch0 = *(volatile unsigned long long*)epoch_ptr;
    // neighbour list of this CTA (nullptr: a grid barrier after every step)
    const int* my_nbr = nbr ? nbr + (size_t)blockIdx.x * kBatchMaxNbr : nullptr;
    unsigned bits = 0;
    constexpr int kLanesX = kTileW / NPT;  // threads along a tile row
    const int r = tid / kLanesX, cx = tid % kLanesX;
    // this CTA's tiles: t0, t0 + stride, ... below t1 (batch_tile_owner)
    int t0, t1, stride;
    if (kBatchStrided) {  // every gridDim.x-th tile: concurrent CTAs work on neighbouring tiles
        t0 = blockIdx.x;
        t1 = ntiles;
        stride = gridDim.x;
    } else {  // a contiguous run: consecutive tiles mostly share a problem
        const int per = (ntiles + gridDim.x - 1) / gridDim.x;
        t0 = blockIdx.x * per;
        t1 = min(ntiles, t0 + per);
        stride = 1;
    }
    // running index k of this CTA's tiles over all steps: stage k & 1,
    // phase parity (k >> 1) & 1
    auto issue = [&](int t, int k, int par) {
        const int4 T = tiles[t];
        stage_T[k & 1] = T;  // read by every thread after the barrier of tile k
        // T.w: the box's bytes, top bit set for a wrapping problem (no load of
        // the problem's record before the copy: its tensor map is addressed)
        const unsigned tw = (unsigned)T.w;
        // the problem's constants come along unless the stage still holds them
        const bool consts = const_of[k & 1] != T.x;
        mbar_arrive_expect_tx(&bar[k & 1], (tw & 0x7fffffffu) + (consts ? (uint32_t)kConstBytes : 0u));
        // array column T.y (interior column T.y - 4), array row T.z (interior row T.z - 1);
        // a wrapping problem's box starts one row lower, at its first interior row
        tma_load_3d(box0 + (k & 1) * kStageFloats, &probs[T.x].tm[par], T.y, 0, T.z + (int)(tw >> 31),
                    &bar[k & 1]);
        if (consts) {
            bulk_g2s(sConst[k & 1], reinterpret_cast<const unsigned char*>(probs + T.x) + kConstOff,
                     (uint32_t)kConstBytes, &bar[k & 1]);
            const_of[k & 1] = T.x;
        }
    };
    auto wait = [&](int k) { return mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), kBatchWaitLimit); };
    int k = 0, issued = -1, waited = -1;
    for (int s = 0; s < nsteps; ++s) {
        const long long level = level0 + s;
        const int par = (int)(level & 1);
        // (a give-up elsewhere is seen in the waits below, by the CTA as a whole)
        if (s > 0 && my_nbr && !wait_neighbours(my_nbr, done, epoch0 + s, status)) return;
        if (t0 < t1) {
            if (tid == 0) issue(t0, k, par);
            issued = k;
        }
        // y ghost rows of such problems are written on the launch's last step only
        const bool last = s == nsteps - 1;
        for (int t = t0; t < t1; t += stride, ++k) {
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
            if (t + stride < t1) {
                if (tid == 0) issue(t + stride, k + 1, par);
                issued = k + 1;
            }
            const int4 T = stage_T[k & 1];
            const BatchProb& P = probs[T.x];
            const Model<float>& sM = *reinterpret_cast<const Model<float>*>(sConst[k & 1]);
            const Grid<float>& sG = *reinterpret_cast<const Grid<float>*>(sConst[k & 1] + kGridInConst);
            // the problem wraps in y inside its tiles
            const bool wrap = (unsigned)T.w >> 31;
            if constexpr (NPT == 1) {
                const int ix = T.y + cx, iy = T.z + r;
                if (ix < sG.nx && iy < sG.ny) {
                    // box row of interior row iy: iy + 1, or iy for a wrapping problem
                    const float* b = box0 + (k & 1) * kStageFloats + (r + !wrap) * kBoxRow + (cx + 4);
                    // north / south offsets in the box: across the periodic edge
                    // of a wrapping problem, the opposite interior row
                    const int dn = wrap && iy == sG.ny - 1 ? -(sG.ny - 1) * kBoxRow : kBoxRow;
                    const int ds = wrap && iy == 0 ? (sG.ny - 1) * kBoxRow : -kBoxRow;
                    float f[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = b[i * kBoxPop];
                    float rho, ux, uy, Tt;
                    moments<float, TM>(f, sM, rho, ux, uy, Tt);
                    bits |= health(rho, ux, uy, Tt);
                    float ofe[9], o[9];
                    relaxation<float, TM>(sM, f, rho, ux, uy, Tt, ofe);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const float* bp = b + i * kBoxPop;
                        o[i] = update(sM, i, ofe[i], f[i], bp[1], bp[-1], bp[dn], bp[ds]);
                    }
                    float* fout = P.f[par ^ 1];
                    const size_t pl = (size_t)sG.plane;
                    const size_t c = cell(sG, ix, iy);
#pragma unroll
                    for (int i = 0; i < 9; ++i) fout[i * pl + c] = o[i];
                    if (wrap && !last) {
                        if (ix == 0 || ix == sG.nx - 1) write_ghosts_x(sG, fout, ix, iy, o, level + 1);
                    } else if (ix == 0 || iy == 0 || ix == sG.nx - 1 || iy == sG.ny - 1) {
                        write_ghosts(sG, fout, ix, iy, o, level + 1);
                    }
                }
            } else {  // two x-adjacent nodes per thread, 8-byte shared loads and stores
                const int ix0 = T.y + 2 * cx, iy = T.z + r;
                if (ix0 < sG.nx && iy < sG.ny) {
                    const int nvalid = min(2, sG.nx - ix0);
                    const float* b = box0 + (k & 1) * kStageFloats + (r + !wrap) * kBoxRow + (2 * cx + 4);
                    const int dn = wrap && iy == sG.ny - 1 ? -(sG.ny - 1) * kBoxRow : kBoxRow;
                    const int ds = wrap && iy == 0 ? (sG.ny - 1) * kBoxRow : -kBoxRow;
                    float2 o[9];
                    bits |= pair_update<TM, false>(sM, b, kBoxPop, dn, ds, nvalid, o);
                    float* fout = P.f[par ^ 1];
                    const size_t pl = (size_t)sG.plane;
                    float* out = fout + cell(sG, ix0, iy);  // 8-byte aligned: ix0 + PADX is even
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (nvalid == 2)
                            *reinterpret_cast<float2*>(out + i * pl) = o[i];
                        else
                            out[i * pl] = o[i].x;
                    }
                    const bool ghost_y = !(wrap && !last);
                    const bool edge_row = ghost_y && (iy == 0 || iy == sG.ny - 1);
                    if (edge_row || ix0 == 0 || ix0 + nvalid == sG.nx) {
                        for (int j = 0; j < nvalid; ++j) {
                            const int ix = ix0 + j;
                            if (!(edge_row || ix == 0 || ix == sG.nx - 1)) continue;
                            float v[9];
#pragma unroll
                            for (int i = 0; i < 9; ++i) v[i] = out[i * pl + j];
                            if (ghost_y)
                                write_ghosts(sG, fout, ix, iy, v, level + 1);
                            else
                                write_ghosts_x(sG, fout, ix, iy, v, level + 1);
                        }
                    }
                }
            }
        }
        if (my_nbr)
            publish_step(done, epoch0 + s + 1);
        else if (!grid_barrier(bar_count, bar_gen, status))
            return;
    }
    // one grid barrier per launch: every CTA has read the level and epoch
    // counters before block 0 advances them
    if (my_nbr && !grid_barrier(bar_count, bar_gen, status)) return;
    report(status, bits);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *level_ptr = level0 + nsteps;
        *epoch_ptr = epoch0 + nsteps;
    }
}
// ------------------------------------------------- temporal blocking
// For batches of thin problems (at most kTbRowsMax rows, no periodic x
// sides) one pass advances a segment of kTbW columns (all rows) by NS steps
// (NS odd) inside shared memory: it loads the level with a halo of NS columns
// on each side (the ghost cells included), then each sub-step j updates the
// columns within NS - 1 - j of the segment and fills the ghost cells of the
// new level there by the same rules as write_ghosts, and the pass stores the
// segment of level + NS, its ghost rows and, at a problem's ends, its ghost
// columns.  NS odd puts level + NS in the other level buffer than the one the
// pass reads, so no CTA overwrites data another is still loading; a grid
// barrier separates passes.  The per-node arithmetic is that of every other
// kernel, so the levels are bit-identical to stepping each problem alone;
// DRAM traffic and grid barriers drop by a factor of NS for a redundant
// update of (NS - 1) columns on each side of a segment.
constexpr int kTbW = 128;
constexpr int kTbThreads = 256;

__host__ __device__ constexpr int tb_width(int ns) { return kTbW + 2 * ns; }

// Value of a ghost cell of the level in buffer B (planes of rows_pitch rows of
// width wb, row 0 = ghost row -1, column 0 = global column xo) for the level
// `level`: pulled from the interior cell the rule makes it from.
__device__ __forceinline__ void tb_ghost(const Grid<float>& G, float* B, int wb, int plane, int xo, int side,
                                         int along, long long level) {
    const int part = side_part(G, side, along, level);
    const int kind = part ? G.kind_hi[side] : G.kind_lo[side];
    int gx, gy, sx, sy;  // ghost cell and its source (global coordinates)
    if (side == S_LEFT || side == S_RIGHT) {
        gy = sy = along;
        gx = side == S_LEFT ? -1 : G.nx;
        sx = side == S_LEFT ? 0 : G.nx - 1;
    } else {
        gx = sx = along;
        gy = side == S_BOTTOM ? -1 : G.ny;
        sy = kind == BC_PERIODIC ? (side == S_BOTTOM ? G.ny - 1 : 0) : (side == S_BOTTOM ? 0 : G.ny - 1);
    }
    float* g = B + (gy + 1) * wb + (gx - xo);
    const float* src = B + (sy + 1) * wb + (sx - xo);
    if (kind == BC_DIRICHLET) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i * plane] = G.feq[side][part][i];
    } else if (kind == BC_REFLECT) {
        const bool xs = side == S_LEFT || side == S_RIGHT;
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i * plane] = src[(xs ? mirror_x(i) : mirror_y(i)) * plane];
    } else {  // outflow copies the adjacent node; periodic (y only) the opposite one
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i * plane] = src[i * plane];
    }
}

#ifndef LBM_TB_MIN_BLOCKS
#define LBM_TB_MIN_BLOCKS 2
#endif

template <int TM>
__global__ void __launch_bounds__(kTbThreads, LBM_TB_MIN_BLOCKS)
    k_batch_tb(const BatchProb* __restrict__ probs, const int4* __restrict__ segs, int nsegs, int nsteps,
               int ns_max, int rows_max, long long* level_ptr, unsigned* bar_count, unsigned* bar_gen,
               unsigned* status) {
    __shared__ Model<float> sM;
    __shared__ Grid<float> sG;
    extern __shared__ __align__(16) float tbuf[];
    const int wb = tb_width(ns_max);
    const int plane = (rows_max + 2) * wb;
    const int tid = threadIdx.x;
    const long long level0 = *(volatile long long*)level_ptr;
    unsigned bits = 0;
    const int per = (nsegs + gridDim.x - 1) / gridDim.x;
    const int g0 = blockIdx.x * per, g1 = min(nsegs, g0 + per);
    int done = 0;
    while (done < nsteps) {
        int n = min(ns_max, nsteps - done);
        if ((n & 1) == 0) --n;  // odd: level + n lies in the other level buffer
        const long long level = level0 + done;
        if (*(volatile unsigned*)status & ST_TIMEOUT) return;
        int cur = -1;
        for (int g = g0; g < g1; ++g) {
            const int4 Sg = segs[g];
            const BatchProb& P = probs[Sg.x];
            __syncthreads();  // the previous segment's buffers and constants are no longer read
            if (Sg.x != cur) {
                copy_words(reinterpret_cast<float*>(&sM), reinterpret_cast<const float*>(&P.M),
                           (int)(sizeof(Model<float>) / sizeof(float)));
                copy_words(reinterpret_cast<int*>(&sG), reinterpret_cast<const int*>(&P.G),
                           (int)(sizeof(Grid<float>) / sizeof(int)));
                cur = Sg.x;
                __syncthreads();
            }
            const int nx = sG.nx, ny = sG.ny;
            const int x0 = Sg.y, xo = x0 - n;  // buffer column 0 is global column xo
            const size_t pl = (size_t)sG.plane;
            float* A = tbuf;
            float* B = tbuf + 9 * plane;
            // load level `level` over columns [max(xo, -1), min(x0 + kTbW + n, nx + 1)), rows -1 .. ny
            {
                const float* fin = P.f[(int)(level & 1)];
                const int xa = max(xo, -1), xb = min(x0 + kTbW + n, nx + 1);
                const int w = xb - xa, rows = ny + 2;
                for (int q = tid; q < 9 * rows * w; q += kTbThreads) {
                    const int i = q / (rows * w), rem = q % (rows * w);
                    const int r = rem / w, x = xa + rem % w;
                    A[i * plane + r * wb + (x - xo)] = __ldcg(fin + i * pl + (size_t)r * sG.row + (x + PADX));
                }
            }
            __syncthreads();
            for (int j = 0; j < n; ++j) {
                const long long lj = level + j;
                const int ca = max(x0 - (n - 1 - j), 0), cb = min(x0 + kTbW + (n - 1 - j), nx);
                const int w = cb - ca;
                for (int q = tid; q < w * ny; q += kTbThreads) {
                    const int y = q / w, x = ca + q % w;
                    const float* c = A + (y + 1) * wb + (x - xo);
                    float f[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = c[i * plane];
                    float rho, ux, uy, Tt;
                    moments<float, TM>(f, sM, rho, ux, uy, Tt);
                    bits |= health(rho, ux, uy, Tt);
                    float ofe[9];
                    relaxation<float, TM>(sM, f, rho, ux, uy, Tt, ofe);
                    float* o = B + (y + 1) * wb + (x - xo);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const float* cp = c + i * plane;
                        o[i * plane] = update(sM, i, ofe[i], f[i], cp[1], cp[-1], cp[wb], cp[-wb]);
                    }
                }
                __syncthreads();
                // ghost cells of level lj + 1 that the next sub-step or the store reads
                for (int q = tid; q < 2 * w; q += kTbThreads)
                    tb_ghost(sG, B, wb, plane, xo, q < w ? S_BOTTOM : S_TOP, ca + (q < w ? q : q - w), lj + 1);
                if (xo <= -1)
                    for (int y = tid; y < ny; y += kTbThreads) tb_ghost(sG, B, wb, plane, xo, S_LEFT, y, lj + 1);
                if (x0 + kTbW + n > nx)
                    for (int y = tid; y < ny; y += kTbThreads) tb_ghost(sG, B, wb, plane, xo, S_RIGHT, y, lj + 1);
                __syncthreads();
                float* t = A;
                A = B;
                B = t;
            }
            // store level `level + n`: the segment's columns with their ghost rows,
            // and the ghost columns at the problem's ends
            {
                float* fout = P.f[(int)((level + n) & 1)];
                const int xa = x0 == 0 ? -1 : x0, xb = x0 + kTbW >= nx ? nx + 1 : x0 + kTbW;
                const int w = xb - xa, rows = ny + 2;
                for (int q = tid; q < 9 * rows * w; q += kTbThreads) {
                    const int i = q / (rows * w), rem = q % (rows * w);
                    const int r = rem / w, x = xa + rem % w;
                    const bool corner = (x < 0 || x >= nx) && (r == 0 || r == rows - 1);
                    if (!corner) fout[i * pl + (size_t)r * sG.row + (x + PADX)] = A[i * plane + r * wb + (x - xo)];
                }
            }
        }
        if (!grid_barrier(bar_count, bar_gen, status)) return;
        done += n;
    }
    report(status, bits);
    if (blockIdx.x == 0 && threadIdx.x == 0) *level_ptr = level0 + nsteps;
}

}  // namespace

bool batch_wraps_in_tile(const Grid<float>& G) { return wraps_in_tile(G, kTileH); }

int batch_tile_owner(int t, int ntiles, int grid) {
    return kBatchStrided ? t % grid : t / ((ntiles + grid - 1) / grid);
}

cudaError_t batch_set_wait_cycles(long long cycles) {
    return cudaMemcpyToSymbol(g_wait_cycles, &cycles, sizeof(cycles));
}

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
                           unsigned* bar_count, unsigned* bar_gen, unsigned* status, const BatchSync& sync,
                           int grid, cudaStream_t st) {
    auto kern = k_batch<TM, NPT>;
    cudaError_t e = allow_smem<k_batch<TM, NPT>>(kBatchSmem);
    if (e != cudaSuccess) return e;
    const int* nbr = sync.nbr;
    unsigned long long* done = sync.done;
    unsigned long long* epoch = sync.epoch;
    void* args[] = {(void*)&probs, (void*)&tiles, (void*)&ntiles, (void*)&nsteps, (void*)&level,
                    (void*)&bar_count, (void*)&bar_gen, (void*)&status, (void*)&nbr, (void*)&done,
                    (void*)&epoch};
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
                         unsigned* bar_count, unsigned* bar_gen, unsigned* status, const BatchSync& sync,
                         int grid, int npt, cudaStream_t st) {
    if (npt == 2)
        return launch_batch_v<TM, 2>(probs, tiles, ntiles, nsteps, level, bar_count, bar_gen, status, sync, grid,
                                     st);
    return launch_batch_v<TM, 1>(probs, tiles, ntiles, nsteps, level, bar_count, bar_gen, status, sync, grid, st);
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
                                          unsigned*, unsigned*, const BatchSync&, int, int, cudaStream_t); \
    template int batch_max_grid<TM>(int);
LBM_BATCH_INST(T_INT32)
LBM_BATCH_INST(T_INT64)
LBM_BATCH_INST(T_DF)
LBM_BATCH_INST(T_CONS)
#undef LBM_BATCH_INST

size_t batch_tb_smem(int ns, int rows_max) {
    return sizeof(float) * 2 * 9 * (size_t)(rows_max + 2) * tb_width(ns);
}

int batch_tb_width() { return kTbW; }

template <int TM>
cudaError_t launch_batch_tb(const BatchProb* probs, const int4* segs, int nsegs, int nsteps, int ns, int rows_max,
                            long long* level, unsigned* bar_count, unsigned* bar_gen, unsigned* status, int grid,
                            cudaStream_t st) {
    auto kern = k_batch_tb<TM>;
    const size_t smem = batch_tb_smem(ns, rows_max);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&probs, (void*)&segs,  (void*)&nsegs,     (void*)&nsteps,  (void*)&ns,
                    (void*)&rows_max, (void*)&level, (void*)&bar_count, (void*)&bar_gen, (void*)&status};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTbThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

template <int TM>
int batch_tb_max_grid(int ns, int rows_max) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = batch_tb_smem(ns, rows_max);
    if (cudaFuncSetAttribute(k_batch_tb<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_tb<TM>, kTbThreads, smem);
    return sms * per_sm;
}

#define LBM_BATCH_TB_INST(TM)                                                                                \
    template cudaError_t launch_batch_tb<TM>(const BatchProb*, const int4*, int, int, int, int, long long*,  \
                                             unsigned*, unsigned*, unsigned*, int, cudaStream_t);            \
    template int batch_tb_max_grid<TM>(int, int);
LBM_BATCH_TB_INST(T_INT32)
LBM_BATCH_TB_INST(T_INT64)
LBM_BATCH_TB_INST(T_DF)
LBM_BATCH_TB_INST(T_CONS)
#undef LBM_BATCH_TB_INST

}  // namespace lbm
