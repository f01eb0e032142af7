// lbm_launch.h -- host-side launchers of the liblbm kernels (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include "lbm_device.cuh"

namespace lbm {

// Raise a kernel's dynamic shared-memory limit once per device (the setting
// persists; calling the runtime for it on every launch costs microseconds
// per step on small grids).  Host threads may race here: the bit mask is
// atomic and a repeated call is harmless.
template <auto Kern>
inline cudaError_t allow_smem(size_t bytes) {
    static std::atomic<unsigned> done{0};  // per kernel: one bit per device ordinal < 32
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned bit = dev >= 0 && dev < 32 ? 1u << dev : 0u;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

// CTAs of one full wave of `Kern` on the current device: SMs x resident CTAs
// per SM at `threads` threads and `smem` bytes of dynamic shared memory.
// Cached per device ordinal (devices may differ in SM count); host threads
// that race to fill an entry all store the same value.
template <auto Kern>
inline int full_wave(int threads, size_t smem) {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < 64;
    if (cached) {
        const int v = cache[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kern, threads, smem);
    const int v = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (cached) cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

// Kernel variant and launch shape of the step (chosen by the host, see
// lbm_tune in lbm.h).
enum StepVariant : int { STEP_SIMPLE = 0, STEP_RING = 1, STEP_VEC = 2, STEP_TILE = 3 };
struct StepConfig {
    int variant = STEP_TILE;  // FP64 always uses STEP_SIMPLE
    int tx = 0;               // ring: columns per CTA (128 or 256); vec: nodes per thread (2 or 4)
    int ring = 0;             // ring: shared-memory row slots (4 or 6; 4 when tx = 128)
    int grid = 0;             // ring, tile: CTAs (0 = SMs x resident CTAs per SM)
    const CUtensorMap* tmap = nullptr;  // tile: tensor map of the input level
};

// Box of the tiled tensor copy of the tile kernel (x, y extent; 9 planes).
void tile_box_dims(int* bx, int* by);

// The step kernel's data movement alone (lbm_probe_tile_copy): level in the
// tensor map -> fout, each node's nine values copied through, no ghosts.
cudaError_t launch_tile_copy(const CUtensorMap& tmap, float* fout, const Grid<float>& G, unsigned* status,
                             cudaStream_t st);

// One step, level `level` in fin -> level + 1 in fout (ghosts included).
// status: 4 words, zero-initialised by the owner: [0] the health bits,
// [2] and [3] the tile kernel's scheduling counters (zero between launches;
// the kernel leaves them so); launches that share a status buffer must not
// overlap.
template <typename S, int TM>
cudaError_t launch_step(const S* fin, S* fout, const Model<S>& M, const Grid<S>& G,
                        long long level, unsigned* status, cudaStream_t st, const StepConfig& cfg);

// f = f^eq(fields) on the interior (fields are ny x nx, storage type).
template <typename S>
cudaError_t launch_init(S* f, const S* rho, const S* ux, const S* uy, const S* T,
                        const Model<S>& M, const Grid<S>& G, cudaStream_t st);

// Fill the ghost layer of f for time level `level` from its interior.
template <typename S>
cudaError_t launch_fill_ghosts(S* f, const Grid<S>& G, long long level, cudaStream_t st);

// Macroscopic fields of f; outputs may be null.  Sets ST_NONPHYSICAL.
template <typename S, int TM>
cudaError_t launch_moments(const S* f, S* rho, S* ux, S* uy, S* T, const Model<S>& M,
                           const Grid<S>& G, unsigned* status, cudaStream_t st);

// FP64 totals of rho, rho u, E into out[4] (device); `partials` holds
// conservation_partials(G) * 4 doubles.
template <typename S>
int conservation_partials(const Grid<S>& G);
template <typename S>
cudaError_t launch_conservation(const S* f, const Model<double>& M, const Grid<S>& G,
                                double* partials, double* out, cudaStream_t st);

// Interior <-> dense 9 x ny x nx copies.
template <typename S>
cudaError_t launch_pack(const S* f, S* dense, const Grid<S>& G, cudaStream_t st);
template <typename S>
cudaError_t launch_unpack(S* f, const S* dense, const Grid<S>& G, cudaStream_t st);

// Adjoint (lbm_adjoint.cu).  a, abar: padded layout; taup: one FP64 slot per
// block (adjoint_partials of them), accumulated across calls.
template <typename S, int TM>
cudaError_t launch_adjoint(const S* f, const S* a, S* abar, const Model<S>& M, const Grid<S>& G,
                           long long level, double* taup, cudaStream_t st);
template <typename S>
int adjoint_partials(const Grid<S>& G);
// FP32 tile adjoint: tmapA over the adjoint level n + 1 (box from
// adjoint_tile_boxes: ax x ay x 9), whose periodic ghost cells must hold the
// wrapped values and whose other ghost cells must be zero; tmapF over the
// forward level n (box fx x fy x 9).  Writes abar's interior and periodic
// ghost cells.
template <int TM>
cudaError_t launch_adjoint_tile(const CUtensorMap& tmapA, const CUtensorMap& tmapF, float* abar,
                                const Model<float>& M, const Grid<float>& G, long long level, double* taup,
                                unsigned* status, cudaStream_t st);
// Periodic ghost cells of an adjoint level from its interior (no-op without
// periodic sides).
cudaError_t launch_adjoint_wrap(float* a, const Grid<float>& G, cudaStream_t st);
void adjoint_tile_boxes(int* ax, int* ay, int* fx, int* fy);
// Seed abar (dense 9 x n) = sum_m qbar_m dq_m/df at the level f; null qbar = 0.
template <typename S, int TM>
cudaError_t launch_moments_vjp(const S* f, const S* qr, const S* qx, const S* qy, const S* qT, S* abar,
                               const Model<S>& M, const Grid<S>& G, cudaStream_t st);
// Field gradient g = sum_i abar_i dF_i/dq at fields q (all dense, n nodes).
template <typename S>
cudaError_t launch_feq_vjp(const S* r, const S* ux, const S* uy, const S* T, const S* abar, S* gr, S* gx,
                           S* gy, S* gT, const Model<S>& M, long long n, cudaStream_t st);

// Batch (lbm_batch.cu): FP32 problems advanced by one cooperative launch.
struct BatchProb {  // 128-byte aligned by its tensor maps
    CUtensorMap tm[2];  // tensor maps of the two levels (box: batch_box_dims, or for
                        // `wrap` problems its interior rows only, x 9)
    float* f[2];        // the two levels; level k lives in f[k & 1]
    Model<float> M;
    Grid<float> G;
    int wrap;           // batch_wraps_in_tile(G): boxes start at the first interior row
    unsigned box_bytes; // bytes of one box
};
// The problem's height fits in one tile row and its y sides are periodic:
// the batch kernel takes the wrapped y neighbours from inside the tile.
bool batch_wraps_in_tile(const Grid<float>& G);
int batch_tile_dims(int* w, int* h);  // returns threads per CTA
void batch_box_dims(int* bx, int* by);
// Step ordering of the batch kernel.  nbr: kBatchMaxNbr CTA indices per CTA
// (-1 padded), the CTAs owning a tile next to one of its own, periodic
// partners included; nullptr orders the steps by a grid barrier instead.
// done: one completed-step counter per CTA; epoch: steps run by the batch so
// far (both only grow).
constexpr int kBatchMaxNbr = 8;
// The CTA of a grid of `grid` that walks tile t of the batch kernel.
int batch_tile_owner(int t, int ntiles, int grid);
// Bound of the batch kernels' inter-CTA waits, in SM cycles (default ~2 s).
cudaError_t batch_set_wait_cycles(long long cycles);
struct BatchSync {
    const int* nbr = nullptr;
    unsigned long long* done = nullptr;
    unsigned long long* epoch = nullptr;
};
// npt: nodes per thread (1: 256-thread CTAs; 2: 128-thread CTAs, two
// x-adjacent nodes each).  grid must not exceed batch_max_grid(npt).
template <int TM>
cudaError_t launch_batch(const BatchProb* probs, const int4* tiles, int ntiles, int nsteps, long long* level,
                         unsigned* bar_count, unsigned* bar_gen, unsigned* status, const BatchSync& sync,
                         int grid, int npt, cudaStream_t st);
template <int TM>
int batch_max_grid(int npt);
// Temporal blocking for thin problems (at most rows_max rows, no periodic x
// sides): segments of batch_tb_width() columns, ns (odd) steps per pass in
// shared memory.  segs: (problem, first column, 0, 0).
constexpr int kBatchTbRowsMax = 8;
int batch_tb_width();
size_t batch_tb_smem(int ns, int rows_max);
template <int TM>
cudaError_t launch_batch_tb(const BatchProb* probs, const int4* segs, int nsegs, int nsteps, int ns, int rows_max,
                            long long* level, unsigned* bar_count, unsigned* bar_gen, unsigned* status, int grid,
                            cudaStream_t st);
template <int TM>
int batch_tb_max_grid(int ns, int rows_max);

// von Neumann scan (lbm_vonneumann.cu): one case is the step's constants
// (folded weights, omega, equilibrium coefficients) and a uniform state.
struct VnCase {
    Model<double> M;
    double rho, ux, uy, T;
};
// J: scratch of 81 doubles per case; radius: ncases x ndirs x nk; growth
// (may be null): ncases.  All device memory.
cudaError_t launch_vn_scan(const VnCase* cases, int ncases, const int2* dirs, int ndirs, int nk, double* J,
                           double* radius, double* growth, cudaStream_t st);

}  // namespace lbm
