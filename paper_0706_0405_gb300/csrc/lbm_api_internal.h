// lbm_api_internal.h -- what the C-ABI sources of liblbm share: the context
// structure, error reporting, the device-allocation wrapper, NVTX ranges,
// derived constants and the tensor-map builders.  Internal to the library.
#pragma once

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_launch.h"

// NVTX ranges around the entry points (header-only NVTX 3: a no-op unless a
// profiler that collects them is attached).
#include <nvtx3/nvToolsExt.h>

using namespace lbm;

struct lbm_ctx {
    int device = 0;
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0, row = 0;  // population and row strides of a level (elements)
    lbm_precision prec = LBM_FP64;
    size_t esize = 8;
    double b = 0, tau = 0, dt = 0, dx = 0;
    lbm_dvm dvm{};
    lbm_dissipation diss{};
    lbm_bc bc[4]{};
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    bool f_owned = true;    // false: f[0], f[1] belong to the caller (lbm_create's f_buf0, f_buf1)
    int cur = 0;            // buffer holding the current level
    long long step = 0;     // step index of the current level
    bool ready = false;     // lbm_init / lbm_set_f / lbm_load done
    unsigned* d_status = nullptr;
    unsigned* h_status = nullptr;
    double* d_partials = nullptr;
    double* d_sums = nullptr;
    double* h_sums = nullptr;
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    Model<double> md{};
    Model<float> mf{};
    Grid<double> gd{};
    Grid<float> gf{};
    StepConfig cfg{};
    CUtensorMap tmap[2];  // FP32: tensor maps of the two level buffers (tile kernel)
    bool tmap_ok = false;
    // adjoint: checkpoints every ck_every steps from level ck_base
    int ck_every = 0;
    long long ck_base = -1;
    std::vector<void*> ck;       // ck[k] holds level ck_base + k * ck_every (padded, with ghosts)
    std::vector<void*> seg;      // recomputed levels of one segment
    void* adj[2] = {nullptr, nullptr};
    // FP32 tile adjoint: tensor maps of the adjoint levels and, per segment
    // level, of its tile (adjoint) and of its halo box (tile recomputation)
    CUtensorMap adj_tmap[2];
    std::vector<CUtensorMap> seg_tmapF, seg_tmapS;
    bool adj_tmaps_ok = false;
    double* d_taup = nullptr;
    double* h_taup = nullptr;
    int ntaup = 0;
    void* d_astage = nullptr;    // staging of the adjoint calls' host arguments
    size_t astage_bytes = 0;
    std::string err;
};

namespace lbm_api {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every device allocation of the library goes through dev_malloc, so that a
// test can make the n-th one fail (lbm_inject_alloc_failure) and check that
// the failure surfaces as LBM_E_NOMEM and leaks nothing.
extern std::atomic<long long> g_alloc_countdown;

template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void**)p, bytes);
}

// message of the last failing lbm_create / lbm_batch_create of this thread
extern thread_local std::string g_create_err;
// record the failure (on the context, else in g_create_err) and return s
lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...);
// LBM_E_NOMEM for an allocation failure, else LBM_E_CUDA
lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
bool finite_pos(double v);
Model<double> build_model(double b, double tau, double dt, double dx, const lbm_dvm& dvm,
                          const lbm_dissipation& diss);
size_t nodes(const lbm_ctx* c);
size_t level_bytes(const lbm_ctx* c);
bool make_tmap_box(CUtensorMap* m, void* base, const lbm_ctx& c, int bx, int by);
bool make_tmap(CUtensorMap* m, void* base, const lbm_ctx& c);
}  // namespace lbm_api

using namespace lbm_api;
