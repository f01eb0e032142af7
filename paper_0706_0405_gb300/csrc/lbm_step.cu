// lbm_step.cu -- the fused time step of the KT D2V9 finite-difference lattice
// Boltzmann scheme with dissipation (Pan, Xu, Zhang & Jiang, IJMPC 2007,
// Eq. SEC-VON-11): moments (Eqs. e4, e5, e7) -> equilibrium (Eqs. e16-e18)
// -> beta-upwind first and central second differences (Eqs. SEC-VON-2a/2b)
// -> BGK relaxation and forward-Euler update, one pass over the grid, with the
// next level's ghost layer written by the edge nodes in the same pass.
#include "lbm_launch.h"
#include "lbm_ptx.cuh"

namespace lbm {

// Probes of an mbarrier before a wait gives up (each probe may suspend the
// thread briefly); far beyond any copy latency.
constexpr uint32_t kWaitLimit = 1u << 22;

// One thread per node.  Each thread reads its node and the four star
// neighbours of all nine populations (the neighbours come from L1/L2: the
// same line serves the adjacent threads), computes the update in registers and
// writes nine values.
template <typename S, int TM>
__global__ void __launch_bounds__(256) k_step_simple(const S* __restrict__ fin, S* __restrict__ fout,
                                                     const Model<S> M, const Grid<S> G,
                                                     long long level, unsigned* status) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= G.nx || iy >= G.ny) return;
    report(status, node_step<S, TM, false>(fin, fout, M, G, ix, iy, level));
}

// ------------------------------------------------- FP32 vectorised kernel
// Each thread updates V x-adjacent nodes of one row (V = 2 or 4), reading the
// nine planes of its row segment and of the rows above and below as V-wide
// vectors, and the two x-neighbours at the ends of the segment as scalars;
// neighbours shared with the adjacent threads come from L1.  This cuts the
// load and address instructions per node by V compared with one node per
// thread, which was the limit of the thread-per-node kernel.  The arithmetic
// per node is the same explicitly rounded sequence (moments, equilibrium,
// update), so the levels are bit-identical to the other variants.
template <int V, int TM>
__global__ void __launch_bounds__(256) k_step_vec(const float* __restrict__ fin, float* __restrict__ fout,
                                                  const Model<float> M, const Grid<float> G,
                                                  long long level, unsigned* status) {
    const int ix0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix0 >= G.nx || iy >= G.ny) return;
    report(status, vec_group<V, TM, false>(fin, fout, M, G, ix0, iy, level));
}

template <int V, int TM>
cudaError_t launch_vec(const float* fin, float* fout, const Model<float>& M, const Grid<float>& G,
                       long long level, unsigned* status, cudaStream_t st) {
    dim3 block(32, 8);
    const int groups = (G.nx + V - 1) / V;
    dim3 grid((groups + block.x - 1) / block.x, (G.ny + block.y - 1) / block.y);
    k_step_vec<V, TM><<<grid, block, 0, st>>>(fin, fout, M, G, level, status);
    return cudaGetLastError();
}

// ------------------------------------------------------ FP32 TMA tile kernel
// Persistent CTAs of 32 x LBM_TILE_Y threads (default 32 x 4) walk
// 64 x LBM_TILE_Y-node tiles.  For each tile one thread issues a single tiled
// tensor copy of the 72 x (LBM_TILE_Y + 2) x 9 box (4 extra columns on each
// side for 16-byte alignment, one extra row above and below, all nine
// planes) into one of two shared-memory stages; the next tile's box is in
// flight while the current one is computed.  Each thread updates two
// x-adjacent nodes (pair_update): it reads their values and those of the
// rows above and below as 8-byte pairs from shared memory, the outer x
// neighbours as single floats, and writes 8-byte pairs.
// CTA j walks tiles j, j + grid, j + 2 grid, ... (static), or claims its
// next tile at run time from a counter in global memory (one atomic per
// tile, one tile ahead of its copy), so that every CTA stays busy until the
// grid runs out of tiles whatever the ratio of tiles to CTAs; the last CTA
// to leave then resets the counter for the next launch.  Waits are bounded:
// on give-up the CTA raises ST_TIMEOUT, lets its copies in flight land and
// leaves.
#ifndef LBM_TILE_X
#define LBM_TILE_X 64
#endif
#ifndef LBM_TILE_Y
#define LBM_TILE_Y 4
#endif
constexpr int kTileX = LBM_TILE_X, kTileY = LBM_TILE_Y;
static_assert(kTileX % 32 == 0, "tile width: a multiple of 32 columns");
constexpr int kTileThreads = (kTileX / 2) * kTileY;
constexpr int kBoxX = kTileX + 8, kBoxY = kTileY + 2;
constexpr int kBoxFloats = kBoxX * kBoxY * 9;
constexpr int kStageFloats = (kBoxFloats + 31) / 32 * 32;  // stages start on 128-byte boundaries

// Shared-memory stages per CTA (boxes in flight + the one being computed) and
// the resident CTAs per SM the register budget is set for: 6 (80 registers)
// in every mode but the double-float one, whose packed update with the
// centre pairs re-read from shared memory fits 72 registers and so 7 CTAs
// (measured on the 4096 x 1024 double Mach reflection: double-float T 69.6
// -> 70.9 GLUPS from 6 to 7 CTAs; FP32 total-energy T 78.1 -> 74.9).
#ifndef LBM_TILE_STAGES
#define LBM_TILE_STAGES 2
#endif
#ifndef LBM_TILE_MIN_BLOCKS
#define LBM_TILE_MIN_BLOCKS 6
#endif
#ifndef LBM_TILE_MIN_BLOCKS_DF
#define LBM_TILE_MIN_BLOCKS_DF 7
#endif
template <int TM>
constexpr int tile_min_blocks() {
    return TM == T_DF ? LBM_TILE_MIN_BLOCKS_DF : LBM_TILE_MIN_BLOCKS;
}
#ifndef LBM_TILE_DYNAMIC
#define LBM_TILE_DYNAMIC 1  // 0: static walk everywhere, 1: as measured below, 2: claims everywhere
#endif
// Tiles claimed at run time (see below) where the grid's CTAs do not divide
// the tiles evenly: with 7 CTAs per SM on the 4096 x 1024 grid (16384 tiles,
// 1064 CTAs) a static walk gives 16 tiles to some CTAs and 15 to others
// (70.9 -> 72.4 GLUPS with run-time claims); with 6 (912 CTAs, 17.96 each)
// the static walk is already even and the claims only cost (78.1 -> 75.7).
template <int TM>
constexpr bool dynamic_tiles() {
    return LBM_TILE_DYNAMIC == 2 || (LBM_TILE_DYNAMIC == 1 && tile_min_blocks<TM>() != LBM_TILE_MIN_BLOCKS);
}
constexpr int kStages = LBM_TILE_STAGES;
static_assert(kStages >= 2 && kStages <= 8, "2 to 8 stages");
constexpr size_t kTileSmem = 128 + sizeof(float) * kStages * kStageFloats + kStages * sizeof(uint64_t);
constexpr int kNoTile = 0x7fffffff;
// 1: each step is launched as a programmatic dependent of the previous
// launch on the stream (its CTAs are scheduled while the previous grid
// drains, and wait for that grid's completion before touching memory).
#ifndef LBM_TILE_PDL
#define LBM_TILE_PDL 1
#endif
// Run-time claims one tile ahead of the copies, the claim's result held in
// a register of thread 0 (1: 75.2 -> 76.2 GLUPS over 400 steps in the
// double-float mode), or each tile claimed just before its copy (0).  (Held
// in shared memory instead, the claim stalls warp 0 right after the copy:
// 73.3.)
#ifndef LBM_TILE_CLAIM_AHEAD
#define LBM_TILE_CLAIM_AHEAD 1
#endif
// Claims ahead are taken only where each CTA walks at least this many tiles
// (chosen at launch): on a small grid a CTA that starts late would still take
// its full share instead of leaving tiles to the CTAs that are free first
// (the Mach-3 2048 x 256 tube, 1.9 tiles a CTA: 12.5 us a step with claims
// ahead, 11.4 without).
constexpr int kClaimAheadTiles = 8;

// status[0]: health bits; status[2], status[3]: the tile counter and the
// count of CTAs that have left (both zero between launches).
template <int TM, bool kClaimAhead>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<TM>())
    k_step_tile(const __grid_constant__ CUtensorMap tmap, float* __restrict__ fout, const Model<float> M,
                const Grid<float> G, long long level, unsigned* status, int tiles_x, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // tensor copies need a 128-byte aligned destination: align the base here
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    float* box = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(float) * kStages * kStageFloats);
    __shared__ int abort_flag;
    __shared__ int tile_of[kStages];  // tile held in each stage (kNoTile: none)
    unsigned ahead = 0;  // run-time claims (thread 0): claimed, copy not yet issued
    unsigned* const counter = status + 2;
    unsigned* const left = status + 3;
    const int tid = threadIdx.x, tx = tid % (kTileX / 2), ty = tid / (kTileX / 2);
    // Launched as a programmatic dependent of the previous step: nothing of
    // the two levels (the previous step writes this step's input and reads
    // its output buffer) or of the counters is touched before the previous
    // grid has completed; the next step may be scheduled from here on, its
    // CTAs taking SM slots as this grid's CTAs leave.
    grid_dependency_wait();
    grid_dependents_launch();
    auto issue = [&](int tile, int stage) {
        const int x0 = (tile % tiles_x) * kTileX, y0 = (tile / tiles_x) * kTileY;
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(sizeof(float) * kBoxFloats));
        // array column x0 is interior column x0 - 4; array row y0 is interior row y0 - 1
        tma_load_3d(box + stage * kStageFloats, &tmap, x0, 0, y0, &bar[stage]);
    };
    constexpr bool kDyn = dynamic_tiles<TM>();
    // the tile of this CTA's local tile k: static walk, or (run-time claims)
    // the one held in k's stage
    auto tile_at = [&](int k) {
        if constexpr (kDyn) {
            return tile_of[k % kStages];
        } else {
            const int t = blockIdx.x + k * gridDim.x;
            return t < ntiles ? t : kNoTile;
        }
    };
    // take the tile of local tile k into its stage and start its copy (thread 0)
    auto claim = [&](int k) {
        const int stage = k % kStages;
        if constexpr (!kDyn) {
            const int t = tile_at(k);
            if (t != kNoTile) issue(t, stage);
            return;
        }
        if constexpr (kClaimAhead) {
            // the tile was claimed one round earlier: its copy starts now; the
            // next claim's atomic is issued after the copy, and its result is
            // first needed a tile later, so its round trip overlaps the tile's
            // arithmetic instead of delaying the copy
            const unsigned t = ahead;
            if (t < (unsigned)ntiles) {
                tile_of[stage] = (int)t;
                issue((int)t, stage);
                ahead = atomicAdd(counter, 1u);
            } else {
                tile_of[stage] = kNoTile;
            }
            return;
        }
        const unsigned t = atomicAdd(counter, 1u);
        if (t < (unsigned)ntiles) {
            tile_of[stage] = (int)t;
            issue((int)t, stage);
        } else {
            tile_of[stage] = kNoTile;
        }
    };
    // local tile k of this CTA lives in stage k % kStages; its phase parity
    // is (k / kStages) & 1
    auto wait = [&](int k) {
        return mbar_wait_bounded(&bar[k % kStages], (uint32_t)((k / kStages) & 1), kWaitLimit);
    };
    if (tid == 0) {
        for (int j = 0; j < kStages; ++j) mbar_init(&bar[j], 1);
        fence_mbar_init();
        abort_flag = 0;
        for (int j = 0; j < kStages; ++j) tile_of[j] = kNoTile;
        if constexpr (kDyn && kClaimAhead) ahead = atomicAdd(counter, 1u);
        for (int j = 0; j < kStages - 1; ++j) claim(j);  // fill all stages but one
    }
    __syncthreads();
    const size_t pl = (size_t)G.plane;
    // the box in shared memory is [row][population][column], like the level
    constexpr int P = kBoxX, R = 9 * kBoxX;  // population and row strides in the box
    unsigned bits = 0;
    int k = 0;
    for (;; ++k) {
        // one thread waits for tile k (the others sleep in the barrier rather
        // than spin); the barrier then also says every thread is done with
        // tile k - 1, whose stage the next copy overwrites
        if (tid == 0 && tile_at(k) != kNoTile && !wait(k)) abort_flag = 1;
        __syncthreads();
        const int t = tile_at(k);
        if (abort_flag || t == kNoTile) break;
        // the stage of tile k - 1 now takes the next tile
        if (tid == 0) claim(k + kStages - 1);
        const int ix0 = (t % tiles_x) * kTileX + 2 * tx, iy = (t / tiles_x) * kTileY + ty;
        if (ix0 >= G.nx || iy >= G.ny) continue;
        const int nvalid = min(2, G.nx - ix0);
        // centre of node ix0 in the box: row ty + 1, column 2 tx + 4 (8-byte aligned)
        const float* b = box + (k % kStages) * kStageFloats + (ty + 1) * R + (2 * tx + 4);
        const size_t c0 = cell(G, ix0, iy);  // 8-byte aligned: ix0 + PADX is even
        float* out = fout + c0;
        float2 o[9];
        bits |= pair_update<TM, packed_pair<TM>(), TM == T_DF>(M, b, P, R, -R, nvalid, o);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (nvalid == 2)
                *reinterpret_cast<float2*>(out + i * pl) = o[i];
            else
                out[i * pl] = o[i].x;
        }
        // edge nodes also write the next level's ghost cells (values read back)
        const bool edge_row = iy == 0 || iy == G.ny - 1;
        if (edge_row || ix0 == 0 || ix0 + nvalid == G.nx) {
            for (int j = 0; j < nvalid; ++j) {
                const int ix = ix0 + j;
                if (!(edge_row || ix == 0 || ix == G.nx - 1)) continue;
                float v[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) v[i] = out[i * pl + j];
                write_ghosts(G, fout, ix, iy, v, level + 1);
            }
        }
    }
    report(status, bits);
    if (tid == 0) {
        if (abort_flag) {
            // let the copies in flight land before the CTA's shared memory
            // goes away: tile k (whose wait gave up) and the tiles claimed
            // after it were issued but not waited for
            for (int j = 0; j < kStages - 1; ++j)
                if (tile_at(k + j) != kNoTile) wait(k + j);
            atomicOr(status, ST_TIMEOUT);
        }
        if constexpr (kDyn) {
            // every claim of this CTA is made; the last CTA out resets the
            // counters for the next launch
            __threadfence();
            if (atomicAdd(left, 1u) == gridDim.x - 1) {
                *counter = 0;
                *left = 0;
                __threadfence();
            }
        }
    }
}

// Data-movement twin of k_step_tile for lbm_probe_tile_copy: the same tile
// walk, the same tensor copies of the halo boxes of one level and the same
// 8-byte stores of the other, no arithmetic (each node's nine values are
// copied through).  Its time is what moving the step kernel's bytes costs
// in this access pattern.
__global__ void __launch_bounds__(kTileThreads, LBM_TILE_MIN_BLOCKS)
    k_tile_copy(const __grid_constant__ CUtensorMap tmap, float* __restrict__ fout, const Grid<float> G,
                unsigned* status, int tiles_x, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    float* box = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(float) * kStages * kStageFloats);
    __shared__ int abort_flag;
    const int tid = threadIdx.x, tx = tid % (kTileX / 2), ty = tid / (kTileX / 2);
    if (tid == 0) {
        for (int j = 0; j < kStages; ++j) mbar_init(&bar[j], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    auto issue = [&](int tile, int stage) {
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(sizeof(float) * kBoxFloats));
        tma_load_3d(box + stage * kStageFloats, &tmap, (tile % tiles_x) * kTileX, 0, (tile / tiles_x) * kTileY,
                    &bar[stage]);
    };
    auto wait = [&](int k) {
        return mbar_wait_bounded(&bar[k % kStages], (uint32_t)((k / kStages) & 1), kWaitLimit);
    };
    int issued = -1, waited = -1;
    for (int j = 0; j < kStages - 1; ++j) {
        const int t = blockIdx.x + j * gridDim.x;
        if (t >= ntiles) break;
        if (tid == 0) issue(t, j);
        issued = j;
    }
    const size_t pl = (size_t)G.plane;
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        if (tid == 0 && !wait(k)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) {
            for (int j = waited + 1; j <= issued; ++j) wait(j);
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        waited = k;
        const int kn = k + kStages - 1, tn = blockIdx.x + kn * gridDim.x;
        if (tn < ntiles) {
            if (tid == 0) issue(tn, kn % kStages);
            issued = kn;
        }
        const int ix0 = (t % tiles_x) * kTileX + 2 * tx, iy = (t / tiles_x) * kTileY + ty;
        if (ix0 >= G.nx || iy >= G.ny) continue;
        const float* b = box + (k % kStages) * kStageFloats + (ty + 1) * (9 * kBoxX) + (2 * tx + 4);
        float* out = fout + cell(G, ix0, iy);
        if (ix0 + 1 < G.nx) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                *reinterpret_cast<float2*>(out + i * pl) = *reinterpret_cast<const float2*>(b + i * kBoxX);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i * pl] = b[i * kBoxX];
        }
    }
}

cudaError_t launch_tile_copy(const CUtensorMap& tmap, float* fout, const Grid<float>& G, unsigned* status,
                             cudaStream_t st) {
    constexpr size_t smem = kTileSmem;
    cudaError_t e = allow_smem<k_tile_copy>(smem);
    if (e != cudaSuccess) return e;
    const int tiles_x = (G.nx + kTileX - 1) / kTileX;
    const int ntiles = tiles_x * ((G.ny + kTileY - 1) / kTileY);
    const int grid = min(ntiles, full_wave<k_tile_copy>(kTileThreads, smem));
    k_tile_copy<<<grid, kTileThreads, smem, st>>>(tmap, fout, G, status, tiles_x, ntiles);
    return cudaGetLastError();
}

void tile_box_dims(int* bx, int* by) {
    *bx = kBoxX;
    *by = kBoxY;
}

template <int TM>
cudaError_t launch_tile(const CUtensorMap& tmap, float* fout, const Model<float>& M, const Grid<float>& G,
                        long long level, unsigned* status, int grid_hint, cudaStream_t st) {
    constexpr size_t smem = kTileSmem;
    // both instances have the same launch bounds, so the same occupancy
    cudaError_t e = allow_smem<k_step_tile<TM, false>>(smem);
    if constexpr (dynamic_tiles<TM>())
        if (e == cudaSuccess) e = allow_smem<k_step_tile<TM, true>>(smem);
    if (e != cudaSuccess) return e;
    const int tiles_x = (G.nx + kTileX - 1) / kTileX;
    const int ntiles = tiles_x * ((G.ny + kTileY - 1) / kTileY);
    int grid = grid_hint;
    if (grid <= 0) grid = full_wave<k_step_tile<TM, false>>(kTileThreads, smem);
    if (grid > ntiles) grid = ntiles;
    auto kern = k_step_tile<TM, false>;
    if constexpr (dynamic_tiles<TM>())
        if (LBM_TILE_CLAIM_AHEAD && ntiles >= kClaimAheadTiles * grid) kern = k_step_tile<TM, true>;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kTileThreads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = LBM_TILE_PDL;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kern, tmap, fout, M, G, level, status, tiles_x, ntiles);
}

// ------------------------------------------------------ FP32 ring kernel
// Each CTA owns TX consecutive columns ("strip") and marches up a contiguous
// run of rows of that strip (the runs of all CTAs tile the flattened
// (strip, row) sequence evenly, so one wave of CTAs covers the grid with no
// tail).  Rows of all nine planes, with 4 extra columns on each side, are
// brought into a ring of R shared-memory slots by bulk asynchronous copies
// (one per plane row) that complete on one mbarrier per slot; thread t keeps
// the rows y-1, y, y+1 of its own column in registers and reads the x
// neighbours of row y from the slot.  Every wait is bounded: on give-up the
// CTA raises ST_TIMEOUT, drains its copies in flight (again bounded) and
// returns.

template <int TX, int R, int TM>
__global__ void __launch_bounds__(TX, 2)
    k_step_ring(const float* __restrict__ fin, float* __restrict__ fout, const Model<float> M,
                const Grid<float> G, long long level, unsigned* status, int rows_per_cta, int nstrips) {
    constexpr int WPAD = TX + 8;  // floats per plane row in a slot: interior columns x0-4 .. x0+TX+3
    extern __shared__ __align__(128) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(float) * R * 9 * WPAD);
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int r = 0; r < R; ++r) mbar_init(&bar[r], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    const size_t pl = (size_t)G.plane;
    const long long total = (long long)nstrips * G.ny;
    const long long w_begin = (long long)blockIdx.x * rows_per_cta;
    const long long w_end = min(w_begin + (long long)rows_per_cta, total);
    long long L = 0;  // row loads issued so far by this CTA (slot = L % R, parity = (L / R) & 1)

    for (long long w = w_begin; w < w_end;) {
        const int strip = (int)(w / G.ny);
        const int y0 = (int)(w % G.ny);
        const int n = (int)min((long long)(G.ny - y0), w_end - w);  // rows computed in this segment
        const int x0 = strip * TX;
        const int ix = x0 + tid;
        const uint32_t bytes = (uint32_t)min(WPAD, G.pitch - x0) * (uint32_t)sizeof(float);
        // load k (0 .. n+1) brings array row y0 + k, i.e. interior row y0 - 1 + k
        auto issue = [&](int k) {
            const long long q = L + k;
            const int slot = (int)(q % R);
            mbar_arrive_expect_tx(&bar[slot], 9u * bytes);
            const float* src = fin + (size_t)(y0 + k) * G.row + x0;
            float* dst = ring + (size_t)slot * 9 * WPAD;
#pragma unroll
            for (int i = 0; i < 9; ++i) bulk_g2s(dst + i * WPAD, src + i * pl, bytes, &bar[slot]);
        };
        auto slot_of = [&](int k) { return ring + (size_t)((L + k) % R) * 9 * WPAD; };
        auto wait = [&](int k) -> bool {
            const long long q = L + k;
            return mbar_wait_bounded(&bar[q % R], (uint32_t)((q / R) & 1), kWaitLimit);
        };
        const int nload = n + 2;
        int issued = min(R, nload);
        __syncthreads();  // the previous segment is done with every slot
        if (tid == 0)
            for (int k = 0; k < issued; ++k) issue(k);

        float S[9], C[9], N[9];
        bool ok = wait(0);
        if (ok) {
            const float* sl = slot_of(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) S[i] = sl[i * WPAD + tid + 4];
        }
        ok = ok && wait(1);
        if (ok) {
            const float* sl = slot_of(1);
#pragma unroll
            for (int i = 0; i < 9; ++i) C[i] = sl[i * WPAD + tid + 4];
        }
        if (!ok) abort_flag = 1;
        int waited = ok ? 2 : 0;

        for (int k = 1; k <= n; ++k) {
            __syncthreads();  // slot of load k-1 is free; abort_flag is visible
            if (abort_flag) {
                // drain the copies this CTA still has in flight, then leave
                for (int q = waited; q < issued; ++q) wait(q);
                if (tid == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
            if (tid == 0 && k - 1 + R < nload) {
                issue(k - 1 + R);
                ++issued;
            } else if (k - 1 + R < nload) {
                ++issued;
            }
            if (!wait(k + 1)) {
                abort_flag = 1;
                continue;
            }
            waited = k + 2;
            const float* sc = slot_of(k);
            const float* sn = slot_of(k + 1);
            const int iy = y0 + k - 1;
            if (ix < G.nx) {
                float f[9], o[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    N[i] = sn[i * WPAD + tid + 4];
                    f[i] = C[i];
                }
                float rho, ux, uy, T;
                moments<float, TM>(f, M, rho, ux, uy, T);
                report(status, health(rho, ux, uy, T));
                float fe[9];
                relaxation<float, TM>(M, f, rho, ux, uy, T, fe);
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    o[i] = update(M, i, fe[i], C[i], sc[i * WPAD + tid + 5], sc[i * WPAD + tid + 3],
                                  N[i], S[i]);
                const size_t c = cell(G, ix, iy);
#pragma unroll
                for (int i = 0; i < 9; ++i) fout[i * pl + c] = o[i];
                if (ix == 0 || iy == 0 || ix == G.nx - 1 || iy == G.ny - 1)
                    write_ghosts(G, fout, ix, iy, o, level + 1);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S[i] = C[i];
                C[i] = N[i];
            }
        }
        __syncthreads();
        if (abort_flag) {
            for (int q = waited; q < issued; ++q) wait(q);
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        L += nload;
        w += n;
    }
}

template <int TX, int R>
constexpr size_t ring_smem_bytes() {
    return sizeof(float) * R * 9 * (TX + 8) + sizeof(uint64_t) * R;
}

template <int TX, int R, int TM>
cudaError_t launch_ring(const float* fin, float* fout, const Model<float>& M, const Grid<float>& G,
                        long long level, unsigned* status, int grid_hint, cudaStream_t st) {
    constexpr size_t smem = ring_smem_bytes<TX, R>();
    auto kern = k_step_ring<TX, R, TM>;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_smem<k_step_ring<TX, R, TM>>(smem);
        if (e != cudaSuccess) return e;
    }
    int grid = grid_hint;
    if (grid <= 0) grid = full_wave<k_step_ring<TX, R, TM>>(TX, smem);
    const int nstrips = (G.nx + TX - 1) / TX;
    const long long total = (long long)nstrips * G.ny;
    const int rows_per_cta = (int)((total + grid - 1) / grid);
    grid = (int)((total + rows_per_cta - 1) / rows_per_cta);
    kern<<<grid, TX, smem, st>>>(fin, fout, M, G, level, status, rows_per_cta, nstrips);
    return cudaGetLastError();
}

template <typename S, int TM>
cudaError_t launch_step(const S* fin, S* fout, const Model<S>& M, const Grid<S>& G,
                        long long level, unsigned* status, cudaStream_t st, const StepConfig& cfg) {
    if constexpr (sizeof(S) == 4) {
        if (cfg.variant == STEP_TILE && cfg.tmap != nullptr)
            return launch_tile<TM>(*cfg.tmap, fout, M, G, level, status, cfg.grid, st);
        if (cfg.variant == STEP_VEC) {
            if (cfg.tx == 2) return launch_vec<2, TM>(fin, fout, M, G, level, status, st);
            return launch_vec<4, TM>(fin, fout, M, G, level, status, st);
        }
        if (cfg.variant == STEP_RING) {
            if (cfg.tx == 128) return launch_ring<128, 4, TM>(fin, fout, M, G, level, status, cfg.grid, st);
            if (cfg.ring == 6) return launch_ring<256, 6, TM>(fin, fout, M, G, level, status, cfg.grid, st);
            return launch_ring<256, 4, TM>(fin, fout, M, G, level, status, cfg.grid, st);
        }
    }
    dim3 block(64, 4);
    dim3 grid((G.nx + block.x - 1) / block.x, (G.ny + block.y - 1) / block.y);
    k_step_simple<S, TM><<<grid, block, 0, st>>>(fin, fout, M, G, level, status);
    return cudaGetLastError();
}

#define LBM_STEP_INST(S, TM)                                                                     \
    template cudaError_t launch_step<S, TM>(const S*, S*, const Model<S>&, const Grid<S>&,        \
                                            long long, unsigned*, cudaStream_t, const StepConfig&);
LBM_STEP_INST(double, T_PLAIN)
LBM_STEP_INST(float, T_INT32)
LBM_STEP_INST(float, T_INT64)
LBM_STEP_INST(float, T_DF)
LBM_STEP_INST(float, T_CONS)
#undef LBM_STEP_INST

}  // namespace lbm
