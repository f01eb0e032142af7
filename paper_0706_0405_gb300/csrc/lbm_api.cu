// lbm_api.cu -- the C ABI of liblbm (declared in include/lbm.h): context
// lifetime, parameter checks, derived constants, buffer management and the
// calls that queue the kernels on the caller's stream.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>
#include <string>

#include "../../include/lbm.h"
#include "lbm_launch.h"

// NVTX ranges around the entry points (header-only NVTX 3: a no-op unless a
// profiler that collects them is attached).
#include <nvtx3/nvToolsExt.h>
namespace {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every device allocation of the library goes through dev_malloc, so that a
// test can make the n-th one fail (lbm_inject_alloc_failure) and check that
// the failure surfaces as LBM_E_NOMEM and leaks nothing.
std::atomic<long long> g_alloc_countdown{-1};

template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void**)p, bytes);
}
}  // namespace

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

namespace {

thread_local std::string g_create_err;

lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_err = buf;
    return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call, what)                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Velocity signs of Eq. (e14) with the diagonals read as c2 (cos, sin).
constexpr int SGX[9] = {0, -1, 0, 1, 0, -1, 1, 1, -1};
constexpr int SGY[9] = {0, 0, -1, 0, 1, -1, -1, 1, 1};

// Derived constants of Eqs. (e16)-(e18) and of the folded update weights of
// Eqs. (SEC-VON-2a/2b, SEC-VON-11), in FP64.
Model<double> build_model(double b, double tau, double dt, double dx, const lbm_dvm& dvm,
                          const lbm_dissipation& diss) {
    Model<double> M{};
    const double c1 = dvm.c1, c2 = dvm.c2, e0 = dvm.eta0;
    const double c1s = c1 * c1, c2s = c2 * c2, e0s = e0 * e0;
    M.omega = dt / tau;
    M.c1 = c1;
    M.d = c2 / std::sqrt(2.0);
    M.c1s = c1s;
    M.c2s = c2s;
    M.eta2 = e0s;
    M.inv_b = 1.0 / b;
    M.b = b;
    M.k0 = (b - 2.0) / e0s;
    const double q1 = 4.0 * (c1s - c2s), q5 = 4.0 * (c2s - c1s);
    M.a1c = -c2s / q1;
    M.a1T = ((b - 2.0) * c2s / e0s + 2.0) / q1;
    M.a1u = (c2s / c1s) / q1;
    M.a5c = -c1s / q5;
    M.a5T = ((b - 2.0) * c1s / e0s + 2.0) / q5;
    M.a5u = (c1s / c2s) / q5;
    const double d1 = 2.0 * c1s * (c1s - c2s), d5 = 2.0 * c2s * (c2s - c1s);
    M.b1c = -c2s / d1;
    M.b1T = (b + 2.0) / d1;
    M.b1u = 1.0 / d1;
    M.b5c = -c1s / d5;
    M.b5T = (b + 2.0) / d5;
    M.b5u = 1.0 / d5;
    M.D1 = 1.0 / (2.0 * c1s * c1s);
    M.D5 = 1.0 / (2.0 * c2s * c2s);
    // moment-exact relaxation: absorb mass / energy defects in the moving set
    // whose c^2 - eta0^2 is larger in size (c1 != c2, so one is nonzero)
    M.h1 = 0.5 / c1;
    const double ea = c1s - e0s, ed = c2s - e0s;
    const bool diag = std::fabs(ed) > std::fabs(ea);
    const double rho_o = diag ? ea / ed : ed / ea;
    M.kcons = 0.25 * rho_o;
    M.kzero = 1.0 - rho_o;
    M.cons_diag = diag ? 1.0 : 0.0;
    const double beta = diss.beta, r = dt / dx;
    for (int i = 0; i < 9; ++i) {
        const double mag = i == 0 ? 0.0 : (i <= 4 ? c1 : M.d);
        const double ax = SGX[i] * mag * r, ay = SGY[i] * mag * r;
        const double mu = diss.lambda[i] * dt / (dx * dx);
        double C = 1.0 - M.omega - 4.0 * mu, E = mu, Wt = mu, N = mu, Sd = mu;
        if (SGX[i] >= 0) {  // Eq. (SEC-VON-2a)
            E -= ax * beta;
            C -= ax * (1.0 - 2.0 * beta);
            Wt += ax * (1.0 - beta);
        } else {            // Eq. (SEC-VON-2b)
            E -= ax * (1.0 - beta);
            C += ax * (1.0 - 2.0 * beta);
            Wt += ax * beta;
        }
        if (SGY[i] >= 0) {
            N -= ay * beta;
            C -= ay * (1.0 - 2.0 * beta);
            Sd += ay * (1.0 - beta);
        } else {
            N -= ay * (1.0 - beta);
            C += ay * (1.0 - 2.0 * beta);
            Sd += ay * beta;
        }
        M.w[i][0] = C;
        M.w[i][1] = E;
        M.w[i][2] = Wt;
        M.w[i][3] = N;
        M.w[i][4] = Sd;
    }
    return M;
}

Model<double> build_model(const lbm_ctx& c) { return build_model(c.b, c.tau, c.dt, c.dx, c.dvm, c.diss); }

void host_equilibrium(const Model<double>& M, double rho, double ux, double uy, double T,
                      double out[9]) {
    const double u2 = ux * ux + uy * uy;
    const double A1 = M.a1c + M.a1T * T + M.a1u * u2, A5 = M.a5c + M.a5T * T + M.a5u * u2;
    const double B1 = M.b1c + M.b1T * T + M.b1u * u2, B5 = M.b5c + M.b5T * T + M.b5u * u2;
    out[0] = rho * M.k0 * T;
    for (int i = 1; i < 9; ++i) {
        const double mag = i <= 4 ? M.c1 : M.d;
        const double vu = SGX[i] * mag * ux + SGY[i] * mag * uy;
        out[i] = i <= 4 ? rho * (A1 + B1 * vu + M.D1 * vu * vu) : rho * (A5 + B5 * vu + M.D5 * vu * vu);
    }
}

template <typename S>
Model<S> cast_model(const Model<double>& d) {
    Model<S> m;
    const double* src = reinterpret_cast<const double*>(&d);
    S* dst = reinterpret_cast<S*>(&m);
    static_assert(sizeof(Model<double>) / sizeof(double) == sizeof(Model<S>) / sizeof(S), "");
    for (size_t k = 0; k < sizeof(Model<double>) / sizeof(double); ++k) dst[k] = (S)src[k];
    return m;
}

template <typename S>
Grid<S> build_grid(const lbm_ctx& c, const Model<double>& M) {
    Grid<S> G{};
    G.nx = c.nx;
    G.ny = c.ny;
    G.pitch = c.pitch;
    G.plane = c.plane;
    G.row = c.row;
    G.dt = c.dt;
    G.dx = c.dx;
    for (int s = 0; s < 4; ++s) {
        G.kind_lo[s] = c.bc[s].kind_lo;
        G.kind_hi[s] = c.bc[s].kind_hi;
        G.split0[s] = c.bc[s].split0;
        G.split_speed[s] = c.bc[s].split_speed;
        G.split_moving[s] = c.bc[s].split_speed != 0.0 ? 1 : 0;
        // first along-index whose cell centre is not below the fixed split
        const int len = (s == LBM_SIDE_LEFT || s == LBM_SIDE_RIGHT) ? c.ny : c.nx;
        int idx = 0;
        while (idx < len && ((double)idx + 0.5) * c.dx < c.bc[s].split0) ++idx;
        G.split_index[s] = idx;
        double lo[9], hi[9];
        const double* a = c.bc[s].state_lo;
        const double* b = c.bc[s].state_hi;
        host_equilibrium(M, a[0], a[1], a[2], a[3], lo);
        host_equilibrium(M, b[0], b[1], b[2], b[3], hi);
        for (int i = 0; i < 9; ++i) {
            G.feq[s][0][i] = (S)lo[i];
            G.feq[s][1][i] = (S)hi[i];
        }
    }
    return G;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

lbm_status validate(int nx, int ny, double b, double tau, double dt, double dx, const lbm_dvm* dvm,
                    const lbm_dissipation* diss, const lbm_bc* bc, lbm_precision prec) {
    if (nx < 1 || ny < 1) return fail(nullptr, LBM_E_INVAL, "nx and ny must be >= 1 (got %d, %d)", nx, ny);
    if (nx > (1 << 24) || ny > (1 << 24)) return fail(nullptr, LBM_E_INVAL, "nx, ny must be <= 2^24");
    if (!finite_pos(b)) return fail(nullptr, LBM_E_INVAL, "b must be finite and > 0");
    if (!finite_pos(tau)) return fail(nullptr, LBM_E_INVAL, "tau must be finite and > 0");
    if (!finite_pos(dt)) return fail(nullptr, LBM_E_INVAL, "dt must be finite and > 0");
    if (!finite_pos(dx)) return fail(nullptr, LBM_E_INVAL, "dx must be finite and > 0");
    if (!dvm || !diss || !bc) return fail(nullptr, LBM_E_INVAL, "dvm, diss and bc must not be NULL");
    if (!finite_pos(dvm->c1) || !finite_pos(dvm->c2) || !finite_pos(dvm->eta0))
        return fail(nullptr, LBM_E_INVAL, "c1, c2 and eta0 must be finite and > 0");
    if (dvm->c1 == dvm->c2)
        return fail(nullptr, LBM_E_INVAL, "c1 == c2 makes the equilibrium singular (Eqs. e17, e18)");
    if (!(diss->beta >= 0.0 && diss->beta <= 0.5))
        return fail(nullptr, LBM_E_INVAL, "beta must lie in [0, 0.5] (got %g)", diss->beta);
    for (int i = 0; i < 9; ++i)
        if (!(std::isfinite(diss->lambda[i]) && diss->lambda[i] >= 0.0))
            return fail(nullptr, LBM_E_INVAL, "lambda[%d] must be finite and >= 0", i);
    if (prec < LBM_FP64 || prec > LBM_FP32_CONS) return fail(nullptr, LBM_E_INVAL, "unknown precision %d", (int)prec);
    for (int s = 0; s < 4; ++s) {
        const lbm_bc& q = bc[s];
        for (int part = 0; part < 2; ++part) {
            const int k = part ? q.kind_hi : q.kind_lo;
            if (k < LBM_BC_PERIODIC || k > LBM_BC_REFLECT)
                return fail(nullptr, LBM_E_INVAL, "side %d: unknown boundary kind %d", s, k);
            if (k == LBM_BC_DIRICHLET) {
                const double* st = part ? q.state_hi : q.state_lo;
                if (!finite_pos(st[0]) || !finite_pos(st[3]) || !std::isfinite(st[1]) || !std::isfinite(st[2]))
                    return fail(nullptr, LBM_E_INVAL, "side %d: Dirichlet state needs rho > 0, T > 0", s);
            }
        }
        if (std::isnan(q.split0) || !std::isfinite(q.split_speed))
            return fail(nullptr, LBM_E_INVAL, "side %d: split0 must not be NaN, split_speed finite", s);
    }
    for (int s = 0; s < 4; s += 2) {
        const bool p0 = bc[s].kind_lo == LBM_BC_PERIODIC || bc[s].kind_hi == LBM_BC_PERIODIC;
        const bool p1 = bc[s + 1].kind_lo == LBM_BC_PERIODIC || bc[s + 1].kind_hi == LBM_BC_PERIODIC;
        if (p0 || p1) {
            const bool ok = bc[s].kind_lo == LBM_BC_PERIODIC && bc[s].kind_hi == LBM_BC_PERIODIC &&
                            bc[s + 1].kind_lo == LBM_BC_PERIODIC && bc[s + 1].kind_hi == LBM_BC_PERIODIC;
            if (!ok)
                return fail(nullptr, LBM_E_INVAL, "periodic sides must come in unsplit opposite pairs");
        }
    }
    return LBM_OK;
}

lbm_status ensure_stage(lbm_ctx* c, size_t bytes) {
    if (c->stage_bytes >= bytes) return LBM_OK;
    if (c->d_stage) cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    LBM_CUDA(c, dev_malloc(&c->d_stage, bytes), "allocating the staging buffer");
    c->stage_bytes = bytes;
    return LBM_OK;
}

lbm_status read_status(lbm_ctx* c) {
    LBM_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
             "reading the status word");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    if (*c->h_status & ST_TIMEOUT) return fail(c, LBM_E_TIMEOUT, "a bounded device wait gave up");
    if (*c->h_status & ST_NONPHYSICAL)
        return fail(c, LBM_E_NONPHYSICAL, "a level had rho <= 0 or a non-finite moment at some node");
    return LBM_OK;
}

lbm_status enter(lbm_ctx* c) {
    if (!c) return fail(nullptr, LBM_E_INVAL, "NULL context");
    LBM_CUDA(c, cudaSetDevice(c->device), "selecting the context's device");
    return LBM_OK;
}

size_t nodes(const lbm_ctx* c) { return (size_t)c->nx * (size_t)c->ny; }

// Typed dispatch on the storage precision / temperature mode.
template <typename F>
cudaError_t dispatch(lbm_ctx* c, F&& fn) {
    switch (c->prec) {
    case LBM_FP64: return fn(double{}, std::integral_constant<int, T_PLAIN>{});
    case LBM_FP32: return fn(float{}, std::integral_constant<int, T_INT32>{});
    case LBM_FP32_T64: return fn(float{}, std::integral_constant<int, T_INT64>{});
    case LBM_FP32_CONS: return fn(float{}, std::integral_constant<int, T_CONS>{});
    default: return fn(float{}, std::integral_constant<int, T_DF>{});
    }
}

template <typename S> const Model<S>& model_of(const lbm_ctx* c);
template <> const Model<double>& model_of<double>(const lbm_ctx* c) { return c->md; }
template <> const Model<float>& model_of<float>(const lbm_ctx* c) { return c->mf; }
template <typename S> const Grid<S>& grid_of(const lbm_ctx* c);
template <> const Grid<double>& grid_of<double>(const lbm_ctx* c) { return c->gd; }
template <> const Grid<float>& grid_of<float>(const lbm_ctx* c) { return c->gf; }

// Copy `bytes` from a host or device pointer into the staging buffer at
// `offset` (returns a device pointer to read from), or pass device pointers
// through.
lbm_status device_view(lbm_ctx* c, const void* p, size_t bytes, size_t offset, const void** out) {
    if (p == nullptr) {
        *out = nullptr;
        return LBM_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return LBM_OK;
    }
    char* dst = static_cast<char*>(c->d_stage) + offset;
    LBM_CUDA(c, cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, c->stream), "copying host input");
    *out = dst;
    return LBM_OK;
}

size_t level_bytes(const lbm_ctx* c) { return (size_t)(c->ny + 2) * (size_t)c->row * c->esize; }

// Keep a copy of the current level (padded, ghosts included) as checkpoint k.
lbm_status save_checkpoint(lbm_ctx* c, size_t k) {
    while (c->ck.size() <= k) {
        void* p = nullptr;
        LBM_CUDA(c, dev_malloc(&p, level_bytes(c)), "allocating a checkpoint");
        c->ck.push_back(p);
    }
    LBM_CUDA(c, cudaMemcpyAsync(c->ck[k], c->f[c->cur], level_bytes(c), cudaMemcpyDeviceToDevice, c->stream),
             "saving a checkpoint");
    return LBM_OK;
}

lbm_status ensure_astage(lbm_ctx* c, size_t bytes) {
    if (c->astage_bytes >= bytes) return LBM_OK;
    cudaFree(c->d_astage);
    c->d_astage = nullptr;
    c->astage_bytes = 0;
    LBM_CUDA(c, dev_malloc(&c->d_astage, bytes), "allocating the adjoint staging buffer");
    c->astage_bytes = bytes;
    return LBM_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// 3D map (x: pitch columns, y: the 9 populations, z: ny + 2 rows) of one
// FP32 level in its row-interleaved layout, with a bx x 9 x by box (in
// shared memory: [row][population][column]).
bool make_tmap_box(CUtensorMap* m, void* base, const lbm_ctx& c, int bx, int by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)c.pitch, 9, (cuuint64_t)(c.ny + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)c.plane * 4, (cuuint64_t)c.row * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, 9, (cuuint32_t)by};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The step kernel's map (tile_box_dims box).
bool make_tmap(CUtensorMap* m, void* base, const lbm_ctx& c) {
    int bx = 0, by = 0;
    tile_box_dims(&bx, &by);
    return make_tmap_box(m, base, c, bx, by);
}


struct CkptHeader {
    char magic[8];
    int nx, ny, prec, esize;
    long long step;
    long long payload;
    char pad[24];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");

}  // namespace

extern "C" lbm_status lbm_probe_tile_copy(int nx, int ny, int reps, double* gbs) {
    if (nx < 1 || ny < 1 || reps < 1 || !gbs) return LBM_E_INVAL;
    lbm_ctx c;  // layout fields only
    c.nx = nx;
    c.ny = ny;
    c.pitch = ((nx + 2 * PADX) + 31) / 32 * 32;
    c.plane = c.pitch;
    c.row = 9LL * c.pitch;
    c.esize = 4;
    const size_t bytes = level_bytes(&c);
    Grid<float> G{};
    G.nx = nx;
    G.ny = ny;
    G.pitch = c.pitch;
    G.plane = c.plane;
    G.row = c.row;
    void* f[2] = {nullptr, nullptr};
    unsigned* status = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status r = LBM_OK;
    CUtensorMap m[2];
    if (dev_malloc(&f[0], bytes) != cudaSuccess || dev_malloc(&f[1], bytes) != cudaSuccess ||
        dev_malloc((void**)&status, sizeof(unsigned)) != cudaSuccess) {
        r = LBM_E_NOMEM;
    } else if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
               cudaMemsetAsync(f[0], 0, bytes, st) != cudaSuccess ||
               cudaMemsetAsync(f[1], 0, bytes, st) != cudaSuccess ||
               cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) {
        r = LBM_E_CUDA;
    } else if (!make_tmap(&m[0], f[0], c) || !make_tmap(&m[1], f[1], c)) {
        r = LBM_E_CUDA;
    } else {
        float best = 1e30f;
        for (int k = 0; k < reps + 2 && r == LBM_OK; ++k) {
            const int a = k & 1;
            if (cudaEventRecord(e0, st) != cudaSuccess ||
                launch_tile_copy(m[a], static_cast<float*>(f[a ^ 1]), G, status, st) != cudaSuccess ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                r = LBM_E_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (k >= 2 && ms < best) best = ms;
        }
        unsigned h = 0;
        if (r == LBM_OK && cudaMemcpy(&h, status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
            r = LBM_E_CUDA;
        if (r == LBM_OK && (h & ST_TIMEOUT)) r = LBM_E_TIMEOUT;
        if (r == LBM_OK) *gbs = 72.0 * (double)nx * (double)ny / (best * 1e-3) / 1e9;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(f[0]);
    cudaFree(f[1]);
    cudaFree(status);
    cudaGetLastError();
    return r;
}

extern "C" {

const char* lbm_version(void) { return "liblbm 0.1 (KT D2V9 FD-LB with dissipation, sm_103a)"; }

const char* lbm_last_error(const lbm_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

lbm_status lbm_create(int nx, int ny, double b, double tau, double dt, double dx, const lbm_dvm* dvm,
                      const lbm_dissipation* diss, const lbm_bc bc[4], lbm_precision prec,
                      void* stream, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_E_INVAL, "out must not be NULL");
    *out = nullptr;
    lbm_status s = validate(nx, ny, b, tau, dt, dx, dvm, diss, bc, prec);
    if (s != LBM_OK) return s;
    lbm_ctx* c = new lbm_ctx();
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, LBM_E_CUDA, "no CUDA device available");
    }
    c->nx = nx;
    c->ny = ny;
    c->pitch = ((nx + 2 * PADX) + 31) / 32 * 32;
    c->plane = c->pitch;
    c->row = 9LL * c->pitch;
    c->prec = prec;
    c->esize = prec == LBM_FP64 ? 8 : 4;
    c->b = b;
    c->tau = tau;
    c->dt = dt;
    c->dx = dx;
    c->dvm = *dvm;
    c->diss = *diss;
    for (int k = 0; k < 4; ++k) c->bc[k] = bc[k];
    c->stream = static_cast<cudaStream_t>(stream);
    if (prec == LBM_FP64) c->cfg = StepConfig{STEP_SIMPLE, 0, 0, 0};
    c->md = build_model(*c);
    c->mf = cast_model<float>(c->md);
    c->gd = build_grid<double>(*c, c->md);
    c->gf = build_grid<float>(*c, c->md);
    const size_t fbytes = level_bytes(c);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = dev_malloc(&c->f[k], fbytes);
    if (e == cudaSuccess) e = dev_malloc((void**)&c->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_status, sizeof(unsigned));
    const int np = c->prec == LBM_FP64 ? conservation_partials(c->gd) : conservation_partials(c->gf);
    if (e == cudaSuccess) e = dev_malloc((void**)&c->d_partials, sizeof(double) * 4 * np);
    if (e == cudaSuccess) e = dev_malloc((void**)&c->d_sums, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_sums, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[0], 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[1], 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) {
        lbm_status r = cuda_fail(nullptr, e, "allocating context buffers");
        lbm_destroy(c);
        return r;
    }
    if (c->prec != LBM_FP64)
        c->tmap_ok = make_tmap(&c->tmap[0], c->f[0], *c) && make_tmap(&c->tmap[1], c->f[1], *c);
    if (c->prec != LBM_FP64 && !c->tmap_ok) c->cfg = StepConfig{STEP_VEC, 4, 0, 0};
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->d_status);
    cudaFreeHost(c->h_status);
    cudaFree(c->d_partials);
    cudaFree(c->d_sums);
    cudaFreeHost(c->h_sums);
    cudaFree(c->d_stage);
    for (void* p : c->ck) cudaFree(p);
    for (void* p : c->seg) cudaFree(p);
    cudaFree(c->adj[0]);
    cudaFree(c->adj[1]);
    cudaFree(c->d_taup);
    cudaFreeHost(c->h_taup);
    cudaFree(c->d_astage);
    cudaGetLastError();
    delete c;
}

lbm_status lbm_init(lbm_ctx* c, const void* rho, const void* ux, const void* uy, const void* T) {
    NvtxRange nvtx_range("lbm_init");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!rho || !ux || !uy || !T) return fail(c, LBM_E_INVAL, "lbm_init: fields must not be NULL");
    const size_t fb = nodes(c) * c->esize;
    if ((s = ensure_stage(c, 9 * fb)) != LBM_OK) return s;
    const void* d[4];
    const void* in[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if ((s = device_view(c, in[k], fb, k * fb, &d[k])) != LBM_OK) return s;
    c->cur = 0;
    c->step = 0;
    c->ck_every = 0;
    c->ck_base = -1;
    LBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "clearing status");
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        S* f = static_cast<S*>(c->f[c->cur]);
        cudaError_t r = launch_init<S>(f, (const S*)d[0], (const S*)d[1], (const S*)d[2], (const S*)d[3],
                                       model_of<S>(c), grid_of<S>(c), c->stream);
        if (r == cudaSuccess) r = launch_fill_ghosts<S>(f, grid_of<S>(c), 0, c->stream);
        return r;
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_init");
    c->ready = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int n) {
    NvtxRange nvtx_range("lbm_step");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (n < 0) return fail(c, LBM_E_INVAL, "lbm_step: n must be >= 0");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_step before lbm_init / lbm_set_f / lbm_load");
    for (int k = 0; k < n; ++k) {
        c->cfg.tmap = c->tmap_ok ? &c->tmap[c->cur] : nullptr;
        cudaError_t e = dispatch(c, [&](auto tag, auto tm) {
            using S = decltype(tag);
            constexpr int TM = decltype(tm)::value;
            return launch_step<S, TM>(static_cast<const S*>(c->f[c->cur]), static_cast<S*>(c->f[c->cur ^ 1]),
                                      model_of<S>(c), grid_of<S>(c), c->step, c->d_status, c->stream, c->cfg);
        });
        if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step");
        c->cur ^= 1;
        c->step += 1;
        if (c->ck_every > 0 && (c->step - c->ck_base) % c->ck_every == 0) {
            const size_t k = (size_t)((c->step - c->ck_base) / c->ck_every);
            lbm_status r = save_checkpoint(c, k);
            if (r != LBM_OK) return r;
        }
    }
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx* c, void* rho, void* ux, void* uy, void* T) {
    NvtxRange nvtx_range("lbm_moments");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_moments before lbm_init");
    const size_t fb = nodes(c) * c->esize;
    void* out[4] = {rho, ux, uy, T};
    void* dev[4];
    bool host_any = false;
    for (int k = 0; k < 4; ++k) {
        if (out[k] && !is_device_ptr(out[k])) host_any = true;
    }
    if (host_any && (s = ensure_stage(c, 9 * fb)) != LBM_OK) return s;
    for (int k = 0; k < 4; ++k)
        dev[k] = !out[k] ? nullptr : is_device_ptr(out[k]) ? out[k] : static_cast<char*>(c->d_stage) + k * fb;
    cudaError_t e = dispatch(c, [&](auto tag, auto tm) {
        using S = decltype(tag);
        constexpr int TM = decltype(tm)::value;
        return launch_moments<S, TM>(static_cast<const S*>(c->f[c->cur]), (S*)dev[0], (S*)dev[1], (S*)dev[2],
                                     (S*)dev[3], model_of<S>(c), grid_of<S>(c), c->d_status, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_moments");
    for (int k = 0; k < 4; ++k)
        if (out[k] && dev[k] != out[k])
            LBM_CUDA(c, cudaMemcpyAsync(out[k], dev[k], fb, cudaMemcpyDeviceToHost, c->stream), "copying moments out");
    if (host_any) return read_status(c);
    return LBM_OK;
}

lbm_status lbm_conservation(lbm_ctx* c, double out[4]) {
    NvtxRange nvtx_range("lbm_conservation");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!out) return fail(c, LBM_E_INVAL, "lbm_conservation: out must not be NULL");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_conservation before lbm_init");
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        return launch_conservation<S>(static_cast<const S*>(c->f[c->cur]), c->md, grid_of<S>(c), c->d_partials,
                                      c->d_sums, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_conservation");
    LBM_CUDA(c, cudaMemcpyAsync(c->h_sums, c->d_sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
             "copying sums");
    s = read_status(c);
    for (int k = 0; k < 4; ++k) out[k] = c->h_sums[k];
    return s;
}

lbm_status lbm_sync(lbm_ctx* c) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    return read_status(c);
}

lbm_status lbm_health(lbm_ctx* c, unsigned* flags) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!flags) return fail(c, LBM_E_INVAL, "lbm_health: flags must not be NULL");
    LBM_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
             "reading the status word");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    *flags = *c->h_status;
    return LBM_OK;
}

lbm_status lbm_get_f(lbm_ctx* c, void* dst) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!dst) return fail(c, LBM_E_INVAL, "lbm_get_f: dst must not be NULL");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_get_f before lbm_init");
    const size_t bytes = 9 * nodes(c) * c->esize;
    const bool dev = is_device_ptr(dst);
    if (!dev && (s = ensure_stage(c, bytes)) != LBM_OK) return s;
    void* target = dev ? dst : c->d_stage;
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        return launch_pack<S>(static_cast<const S*>(c->f[c->cur]), (S*)target, grid_of<S>(c), c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_f");
    if (!dev) {
        LBM_CUDA(c, cudaMemcpyAsync(dst, c->d_stage, bytes, cudaMemcpyDeviceToHost, c->stream), "copying f out");
        LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    }
    return LBM_OK;
}

lbm_status lbm_set_f(lbm_ctx* c, const void* src, long long step) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!src) return fail(c, LBM_E_INVAL, "lbm_set_f: src must not be NULL");
    if (step < 0) return fail(c, LBM_E_INVAL, "lbm_set_f: step must be >= 0");
    const size_t bytes = 9 * nodes(c) * c->esize;
    if (!is_device_ptr(src) && (s = ensure_stage(c, bytes)) != LBM_OK) return s;
    const void* d;
    if ((s = device_view(c, src, bytes, 0, &d)) != LBM_OK) return s;
    LBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "clearing status");
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        S* f = static_cast<S*>(c->f[c->cur]);
        cudaError_t r = launch_unpack<S>(f, (const S*)d, grid_of<S>(c), c->stream);
        if (r == cudaSuccess) r = launch_fill_ghosts<S>(f, grid_of<S>(c), step, c->stream);
        return r;
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_f");
    c->step = step;
    c->ready = true;
    c->ck_every = 0;
    c->ck_base = -1;
    return LBM_OK;
}

long long lbm_step_count(const lbm_ctx* c) { return c ? c->step : -1; }

lbm_status lbm_record(lbm_ctx* c, int every) {
    NvtxRange nvtx_range("lbm_record");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (every < 0) return fail(c, LBM_E_INVAL, "lbm_record: every must be >= 0");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_record before lbm_init");
    c->ck_every = every;
    c->ck_base = every > 0 ? c->step : -1;
    if (every == 0) return LBM_OK;
    return save_checkpoint(c, 0);
}

lbm_status lbm_adjoint_seed(lbm_ctx* c, const void* qr, const void* qx, const void* qy, const void* qT,
                            void* abar) {
    NvtxRange nvtx_range("lbm_adjoint_seed");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!abar) return fail(c, LBM_E_INVAL, "lbm_adjoint_seed: abar must not be NULL");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_adjoint_seed before lbm_init");
    const size_t fb = nodes(c) * c->esize;
    if ((s = ensure_astage(c, 13 * fb)) != LBM_OK) return s;
    const void* in[4] = {qr, qx, qy, qT};
    const void* d[4];
    for (int k = 0; k < 4; ++k) {
        if (!in[k] || is_device_ptr(in[k])) {
            d[k] = in[k];
        } else {
            char* dst = static_cast<char*>(c->d_astage) + (9 + k) * fb;
            LBM_CUDA(c, cudaMemcpyAsync(dst, in[k], fb, cudaMemcpyHostToDevice, c->stream), "copying host qbar");
            d[k] = dst;
        }
    }
    const bool dev_out = is_device_ptr(abar);
    void* out = dev_out ? abar : c->d_astage;
    cudaError_t e = dispatch(c, [&](auto tag, auto tm) {
        using S = decltype(tag);
        constexpr int TM = decltype(tm)::value;
        return launch_moments_vjp<S, TM>(static_cast<const S*>(c->f[c->cur]), (const S*)d[0], (const S*)d[1],
                                         (const S*)d[2], (const S*)d[3], (S*)out, model_of<S>(c), grid_of<S>(c),
                                         c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint_seed");
    if (!dev_out) {
        LBM_CUDA(c, cudaMemcpyAsync(abar, c->d_astage, 9 * fb, cudaMemcpyDeviceToHost, c->stream), "copying abar out");
        LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    }
    return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_ctx* c, int n, void* abar, double* dL_dtau) {
    NvtxRange nvtx_range("lbm_adjoint_step");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!abar || n < 0) return fail(c, LBM_E_INVAL, "lbm_adjoint_step: abar must not be NULL, n >= 0");
    if (c->ck_every <= 0) return fail(c, LBM_E_STATE, "lbm_adjoint_step needs lbm_record first");
    if (c->step - n < c->ck_base)
        return fail(c, LBM_E_INVAL, "lbm_adjoint_step: only %lld steps recorded before the current level",
                    c->step - c->ck_base);
    if (n == 0) return LBM_OK;
    const size_t fb = nodes(c) * c->esize, lb = level_bytes(c);
    const bool fp32 = c->prec != LBM_FP64;
    int abx = 0, aby = 0, afx = 0, afy = 0;
    adjoint_tile_boxes(&abx, &aby, &afx, &afy);
    for (int k = 0; k < 2; ++k)
        if (!c->adj[k]) {
            LBM_CUDA(c, dev_malloc(&c->adj[k], lb), "allocating adjoint levels");
            LBM_CUDA(c, cudaMemsetAsync(c->adj[k], 0, lb, c->stream), "clearing adjoint levels");
            if (k == 1)
                c->adj_tmaps_ok = fp32 && make_tmap_box(&c->adj_tmap[0], c->adj[0], *c, abx, aby) &&
                                  make_tmap_box(&c->adj_tmap[1], c->adj[1], *c, abx, aby);
        }
    while ((int)c->seg.size() < c->ck_every) {
        void* p = nullptr;
        LBM_CUDA(c, dev_malloc(&p, lb), "allocating segment levels");
        c->seg.push_back(p);
        CUtensorMap mf{}, ms{};
        if (c->adj_tmaps_ok && !(make_tmap_box(&mf, p, *c, afx, afy) && make_tmap(&ms, p, *c)))
            c->adj_tmaps_ok = false;
        c->seg_tmapF.push_back(mf);
        c->seg_tmapS.push_back(ms);
    }
    // the tile adjoint (and tile recomputation) with the tile step kernel
    const bool tile = c->adj_tmaps_ok && c->cfg.variant == STEP_TILE;
    const int np = c->prec == LBM_FP64 ? adjoint_partials(c->gd) : adjoint_partials(c->gf);
    if (c->ntaup < np) {
        cudaFree(c->d_taup);
        cudaFreeHost(c->h_taup);
        c->d_taup = nullptr;
        c->h_taup = nullptr;
        LBM_CUDA(c, dev_malloc((void**)&c->d_taup, sizeof(double) * np), "allocating tau partials");
        LBM_CUDA(c, cudaMallocHost((void**)&c->h_taup, sizeof(double) * np), "allocating tau partials");
        c->ntaup = np;
    }
    LBM_CUDA(c, cudaMemsetAsync(c->d_taup, 0, sizeof(double) * np, c->stream), "clearing tau partials");
    // bring the caller's adjoint (dense) into adj[0]
    const bool dev = is_device_ptr(abar);
    if (!dev) {
        if ((s = ensure_astage(c, 13 * fb)) != LBM_OK) return s;
        LBM_CUDA(c, cudaMemcpyAsync(c->d_astage, abar, 9 * fb, cudaMemcpyHostToDevice, c->stream), "copying abar in");
    }
    const void* dense_in = dev ? abar : c->d_astage;
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        return launch_unpack<S>(static_cast<S*>(c->adj[0]), (const S*)dense_in, grid_of<S>(c), c->stream);
    });
    if (e == cudaSuccess && tile) e = launch_adjoint_wrap(static_cast<float*>(c->adj[0]), c->gf, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint_step: unpacking abar");
    StepConfig rcfg = c->cfg;  // recomputation reads segment buffers through their own tensor maps
    if (rcfg.variant == STEP_TILE && !tile) rcfg = StepConfig{STEP_SIMPLE, 0, 0, 0};
    int ac = 0;
    long long L = c->step;
    const long long target = c->step - n;
    long long c0 = L;
    while (L > target) {
        const long long k = (L - 1 - c->ck_base) / c->ck_every;
        c0 = c->ck_base + k * c->ck_every;
        const long long lo = c0 > target ? c0 : target;
        LBM_CUDA(c, cudaMemcpyAsync(c->seg[0], c->ck[(size_t)k], lb, cudaMemcpyDeviceToDevice, c->stream),
                 "restoring a checkpoint");
        for (long long l = c0; l < L - 1; ++l) {
            if (tile) rcfg.tmap = &c->seg_tmapS[(size_t)(l - c0)];
            e = dispatch(c, [&](auto tag, auto tm) {
                using S = decltype(tag);
                constexpr int TM = decltype(tm)::value;
                return launch_step<S, TM>(static_cast<const S*>(c->seg[(size_t)(l - c0)]),
                                          static_cast<S*>(c->seg[(size_t)(l - c0 + 1)]), model_of<S>(c),
                                          grid_of<S>(c), l, c->d_status, c->stream, rcfg);
            });
            if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint_step: recomputing");
        }
        for (long long l = L - 1; l >= lo; --l) {
            e = dispatch(c, [&](auto tag, auto tm) {
                using S = decltype(tag);
                constexpr int TM = decltype(tm)::value;
                if constexpr (std::is_same<S, float>::value) {
                    if (tile)
                        return launch_adjoint_tile<TM>(c->adj_tmap[ac], c->seg_tmapF[(size_t)(l - c0)],
                                                       static_cast<float*>(c->adj[ac ^ 1]), model_of<S>(c),
                                                       grid_of<S>(c), l, c->d_taup, c->d_status, c->stream);
                }
                return launch_adjoint<S, TM>(static_cast<const S*>(c->seg[(size_t)(l - c0)]),
                                             static_cast<const S*>(c->adj[ac]), static_cast<S*>(c->adj[ac ^ 1]),
                                             model_of<S>(c), grid_of<S>(c), l, c->d_taup, c->stream);
            });
            if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint_step");
            ac ^= 1;
        }
        L = lo;
    }
    // the forward state moves back to level `target`
    LBM_CUDA(c, cudaMemcpyAsync(c->f[c->cur], c->seg[(size_t)(target - c0)], lb, cudaMemcpyDeviceToDevice,
                                c->stream),
             "restoring the forward level");
    c->step = target;
    void* dense_out = dev ? abar : c->d_astage;
    e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        return launch_pack<S>(static_cast<const S*>(c->adj[ac]), (S*)dense_out, grid_of<S>(c), c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint_step: packing abar");
    if (!dev)
        LBM_CUDA(c, cudaMemcpyAsync(abar, c->d_astage, 9 * fb, cudaMemcpyDeviceToHost, c->stream), "copying abar out");
    LBM_CUDA(c, cudaMemcpyAsync(c->h_taup, c->d_taup, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream),
             "copying tau partials");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    if (dL_dtau) {
        double t = 0.0;
        for (int b = 0; b < np; ++b) t += c->h_taup[b];
        *dL_dtau += -(c->dt / (c->tau * c->tau)) * t;
    }
    return LBM_OK;
}

lbm_status lbm_feq_vjp(lbm_ctx* c, const void* rho, const void* ux, const void* uy, const void* T,
                       const void* abar, void* grho, void* gux, void* guy, void* gT) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!rho || !ux || !uy || !T || !abar) return fail(c, LBM_E_INVAL, "lbm_feq_vjp: NULL input");
    const size_t fb = nodes(c) * c->esize;
    if ((s = ensure_astage(c, 17 * fb)) != LBM_OK) return s;
    char* st = static_cast<char*>(c->d_astage);
    const void* in[5] = {rho, ux, uy, T, abar};
    const size_t sz[5] = {fb, fb, fb, fb, 9 * fb};
    const size_t off[5] = {0, fb, 2 * fb, 3 * fb, 4 * fb};
    const void* d[5];
    for (int k = 0; k < 5; ++k) {
        if (is_device_ptr(in[k])) {
            d[k] = in[k];
        } else {
            LBM_CUDA(c, cudaMemcpyAsync(st + off[k], in[k], sz[k], cudaMemcpyHostToDevice, c->stream), "copying inputs");
            d[k] = st + off[k];
        }
    }
    void* outs[4] = {grho, gux, guy, gT};
    void* dout[4];
    bool host_any = false;
    for (int k = 0; k < 4; ++k) {
        const bool h = outs[k] && !is_device_ptr(outs[k]);
        host_any |= h;
        dout[k] = !outs[k] ? nullptr : (h ? static_cast<void*>(st + (13 + k) * fb) : outs[k]);
    }
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        return launch_feq_vjp<S>((const S*)d[0], (const S*)d[1], (const S*)d[2], (const S*)d[3], (const S*)d[4],
                                 (S*)dout[0], (S*)dout[1], (S*)dout[2], (S*)dout[3], model_of<S>(c),
                                 (long long)nodes(c), c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_feq_vjp");
    for (int k = 0; k < 4; ++k)
        if (outs[k] && dout[k] != outs[k])
            LBM_CUDA(c, cudaMemcpyAsync(outs[k], dout[k], fb, cudaMemcpyDeviceToHost, c->stream), "copying grads out");
    if (host_any) LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_ctx* c, const lbm_launch* l) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!l) return fail(c, LBM_E_INVAL, "lbm_set_launch: launch must not be NULL");
    if (l->variant != STEP_SIMPLE && l->variant != STEP_RING && l->variant != STEP_VEC && l->variant != STEP_TILE)
        return fail(c, LBM_E_INVAL, "lbm_set_launch: unknown variant %d", l->variant);
    if (l->variant == STEP_TILE) {
        if (c->prec == LBM_FP64) return fail(c, LBM_E_INVAL, "lbm_set_launch: variant 3 is FP32-only");
        if (!c->tmap_ok) return fail(c, LBM_E_INVAL, "lbm_set_launch: tensor maps unavailable on this driver");
        if (l->grid < 0) return fail(c, LBM_E_INVAL, "lbm_set_launch: grid must be >= 0");
    }
    if (l->variant == STEP_VEC) {
        if (c->prec == LBM_FP64) return fail(c, LBM_E_INVAL, "lbm_set_launch: variant 2 is FP32-only");
        if (l->tx != 2 && l->tx != 4) return fail(c, LBM_E_INVAL, "lbm_set_launch: variant 2 needs tx = 2 or 4");
    }
    if (l->variant == STEP_RING) {
        if (c->prec == LBM_FP64) return fail(c, LBM_E_INVAL, "lbm_set_launch: variant 1 is FP32-only");
        const bool ok = (l->tx == 256 && (l->ring == 4 || l->ring == 6)) || (l->tx == 128 && l->ring == 4);
        if (!ok) return fail(c, LBM_E_INVAL, "lbm_set_launch: tx/ring must be 256/4, 256/6 or 128/4");
        if (l->grid < 0) return fail(c, LBM_E_INVAL, "lbm_set_launch: grid must be >= 0");
    }
    c->cfg.variant = l->variant;
    c->cfg.tx = l->tx;
    c->cfg.ring = l->ring;
    c->cfg.grid = l->grid;
    return LBM_OK;
}

lbm_status lbm_get_launch(const lbm_ctx* c, lbm_launch* l) {
    if (!c || !l) return fail(nullptr, LBM_E_INVAL, "lbm_get_launch: NULL argument");
    l->variant = c->cfg.variant;
    l->tx = c->cfg.tx;
    l->ring = c->cfg.ring;
    l->grid = c->cfg.grid;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx* c, int steps, lbm_launch* best, double* ms, int* n_candidates) {
    NvtxRange nvtx_range("lbm_autotune");
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (steps < 1) return fail(c, LBM_E_INVAL, "lbm_autotune: steps must be >= 1");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_autotune before lbm_init");
    lbm_launch cands[8];
    int nc = 0;
    cands[nc++] = {STEP_SIMPLE, 0, 0, 0};
    if (c->prec != LBM_FP64) {
        if (c->tmap_ok) cands[nc++] = {STEP_TILE, 0, 0, 0};
        cands[nc++] = {STEP_VEC, 4, 0, 0};
        cands[nc++] = {STEP_VEC, 2, 0, 0};
        cands[nc++] = {STEP_RING, 256, 4, 0};
        cands[nc++] = {STEP_RING, 256, 6, 0};
        cands[nc++] = {STEP_RING, 128, 4, 0};
    }
    // save the state (interior via the staging buffer, step counter, flags)
    const size_t bytes = 9 * nodes(c) * c->esize;
    if ((s = ensure_stage(c, bytes)) != LBM_OK) return s;
    const long long step0 = c->step;
    const StepConfig cfg0 = c->cfg;
    const int every0 = c->ck_every;
    c->ck_every = 0;  // trial steps must not overwrite recorded checkpoints
    cudaError_t e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        return launch_pack<S>(static_cast<const S*>(c->f[c->cur]), (S*)c->d_stage, grid_of<S>(c), c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_autotune: saving the state");
    LBM_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
             "lbm_autotune: saving the flags");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream), "lbm_autotune");
    const unsigned flags0 = *c->h_status;
    cudaEvent_t ev[2];
    LBM_CUDA(c, cudaEventCreate(&ev[0]), "lbm_autotune: events");
    LBM_CUDA(c, cudaEventCreate(&ev[1]), "lbm_autotune: events");
    int bi = -1;
    float bt = 0.0f;
    lbm_status r = LBM_OK;
    for (int k = 0; k < nc && r == LBM_OK; ++k) {
        c->cfg = StepConfig{cands[k].variant, cands[k].tx, cands[k].ring, cands[k].grid};
        if ((r = lbm_step(c, 1)) != LBM_OK) break;
        cudaEventRecord(ev[0], c->stream);
        if ((r = lbm_step(c, steps)) != LBM_OK) break;
        cudaEventRecord(ev[1], c->stream);
        if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
            r = fail(c, LBM_E_CUDA, "lbm_autotune: timing failed");
            break;
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (ms) ms[k] = t / steps;
        if (bi < 0 || t < bt) {
            bi = k;
            bt = t;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    // restore the state whatever happened
    e = dispatch(c, [&](auto tag, auto) {
        using S = decltype(tag);
        S* f = static_cast<S*>(c->f[c->cur]);
        cudaError_t q = launch_unpack<S>(f, (const S*)c->d_stage, grid_of<S>(c), c->stream);
        if (q == cudaSuccess) q = launch_fill_ghosts<S>(f, grid_of<S>(c), step0, c->stream);
        return q;
    });
    c->step = step0;
    c->ck_every = every0;
    *c->h_status = flags0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_status, c->h_status, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_autotune: restoring the state");
    if (r != LBM_OK) {
        c->cfg = cfg0;
        return r;
    }
    c->cfg = StepConfig{cands[bi].variant, cands[bi].tx, cands[bi].ring, cands[bi].grid};
    if (best) *best = cands[bi];
    if (n_candidates) *n_candidates = nc;
    return LBM_OK;
}

size_t lbm_checkpoint_bytes(const lbm_ctx* c) {
    return c ? sizeof(CkptHeader) + 9 * nodes(c) * c->esize : 0;
}

lbm_status lbm_save(lbm_ctx* c, void* buf, size_t bytes) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!buf || bytes < lbm_checkpoint_bytes(c))
        return fail(c, LBM_E_INVAL, "lbm_save: buffer must hold lbm_checkpoint_bytes() bytes");
    if (!c->ready) return fail(c, LBM_E_STATE, "lbm_save before lbm_init");
    CkptHeader h{};
    std::memcpy(h.magic, "KTLBMCK1", 8);
    h.nx = c->nx;
    h.ny = c->ny;
    h.prec = (int)c->prec;
    h.esize = (int)c->esize;
    h.step = c->step;
    h.payload = (long long)(9 * nodes(c) * c->esize);
    char* p = static_cast<char*>(buf);
    if (is_device_ptr(buf)) {
        LBM_CUDA(c, cudaMemcpyAsync(p, &h, sizeof h, cudaMemcpyHostToDevice, c->stream), "writing header");
        if ((s = lbm_get_f(c, p + sizeof h)) != LBM_OK) return s;
        LBM_CUDA(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
        return LBM_OK;
    }
    std::memcpy(p, &h, sizeof h);
    return lbm_get_f(c, p + sizeof h);
}

lbm_status lbm_load(lbm_ctx* c, const void* buf, size_t bytes) {
    lbm_status s = enter(c);
    if (s != LBM_OK) return s;
    if (!buf || bytes < sizeof(CkptHeader)) return fail(c, LBM_E_INVAL, "lbm_load: buffer too small");
    CkptHeader h{};
    const char* p = static_cast<const char*>(buf);
    if (is_device_ptr(buf))
        LBM_CUDA(c, cudaMemcpy(&h, p, sizeof h, cudaMemcpyDeviceToHost), "reading header");
    else
        std::memcpy(&h, p, sizeof h);
    if (std::memcmp(h.magic, "KTLBMCK1", 8) != 0 || h.nx != c->nx || h.ny != c->ny || h.prec != (int)c->prec ||
        h.payload != (long long)(9 * nodes(c) * c->esize) || bytes < lbm_checkpoint_bytes(c) || h.step < 0)
        return fail(c, LBM_E_INVAL, "lbm_load: checkpoint does not match this context");
    return lbm_set_f(c, p + sizeof h, h.step);
}

}  // extern "C"

// ------------------------------------------------------------------ batch
struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    lbm_precision prec = LBM_FP32;
    cudaStream_t stream = nullptr;
    int device = 0;
    BatchProb* d_probs = nullptr;
    int4* d_tiles = nullptr;
    int ntiles = 0;
    std::vector<int4> tiles;           // host copy of the tile list
    std::vector<int> tiles_x, tiles_y, tile_base;   // per problem
    std::vector<char> periodic_x, periodic_y;       // per problem (any part of a side)
    // step ordering of the tile kernel: neighbour lists for grid nbr_grid
    int* d_nbr = nullptr;
    unsigned long long* d_done = nullptr;
    unsigned long long* d_epoch = nullptr;
    int nbr_cap = 0;    // CTAs the arrays hold
    int nbr_grid = -1;  // grid the lists were made for
    bool nbr_ok = false;
    long long* d_level = nullptr;
    unsigned* d_bar = nullptr;     // [0] arrivals, [1] generation
    unsigned* d_status = nullptr;
    unsigned* h_status = nullptr;
    long long step = 0;
    bool ready = false;
    int grid = 0;
    int npt = 1;                  // nodes per thread of the batch kernel (1 or 2)
    int max_grid[3] = {0, 0, 0};  // resident CTAs of a full wave, per npt
    int block = 0;                // steps per pass of the temporal-blocking kernel (0: tile kernel)
    bool tb_ok = false;           // every problem thin enough, none periodic in x
    int rows_max = 0;
    int4* d_segs = nullptr;
    int nsegs = 0;
    int tb_max_grid[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // per odd steps-per-pass 3, 5, 7
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_n = -1;
    int graph_state = 0;          // 1 captured and replayed, -1 capture failed
    cudaStream_t gstream = nullptr;  // private stream the graph runs on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::string err;
};

namespace {
lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& msg) {
    if (b) b->err = msg;
    else g_create_err = msg;
    return s;
}

// For each CTA of a grid, the other CTAs owning a tile next to one of its
// tiles in x or y, across periodic sides too.  False if some CTA has more
// than kBatchMaxNbr.
bool batch_neighbour_lists(const lbm_batch* b, int grid, std::vector<int>& out) {
    out.assign((size_t)grid * kBatchMaxNbr, -1);
    std::vector<int> cnt(grid, 0);
    auto add = [&](int c, int n) {
        if (n == c) return true;
        for (int j = 0; j < cnt[c]; ++j)
            if (out[(size_t)c * kBatchMaxNbr + j] == n) return true;
        if (cnt[c] == kBatchMaxNbr) return false;
        out[(size_t)c * kBatchMaxNbr + cnt[c]++] = n;
        return true;
    };
    int tw = 0, th = 0;
    batch_tile_dims(&tw, &th);
    for (int t = 0; t < b->ntiles; ++t) {
        const int4 T = b->tiles[t];
        const int p = T.x, tx = b->tiles_x[p], ty = b->tiles_y[p];
        const int ix = T.y / tw, iy = T.z / th, c = batch_tile_owner(t, b->ntiles, grid);
        const int nb[4][2] = {{ix - 1, iy}, {ix + 1, iy}, {ix, iy - 1}, {ix, iy + 1}};
        for (const auto& q : nb) {
            int jx = q[0], jy = q[1];
            if (jx < 0 || jx >= tx) {
                if (!b->periodic_x[p]) continue;
                jx = (jx + tx) % tx;
            }
            if (jy < 0 || jy >= ty) {
                if (!b->periodic_y[p]) continue;
                jy = (jy + ty) % ty;
            }
            if (!add(c, batch_tile_owner(b->tile_base[p] + jy * tx + jx, b->ntiles, grid))) return false;
        }
    }
    return true;
}

// Make the neighbour lists match the current grid (outside graph capture:
// waits for the stream, then copies synchronously).
cudaError_t batch_prepare_sync(lbm_batch* b) {
    if (b->block > 1 || b->nbr_grid == b->grid) return cudaSuccess;
    std::vector<int> lists;
    b->nbr_ok = b->grid <= b->nbr_cap && batch_neighbour_lists(b, b->grid, lists);
    b->nbr_grid = b->grid;
    if (!b->nbr_ok) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_nbr, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) b->nbr_ok = false;
    return e;
}

cudaError_t batch_launch(lbm_batch* b, int n) {
    auto go = [&](auto tm) {
        constexpr int TM = decltype(tm)::value;
        if (b->block > 1)
            return launch_batch_tb<TM>(b->d_probs, b->d_segs, b->nsegs, n, b->block, b->rows_max, b->d_level,
                                       b->d_bar, b->d_bar + 1, b->d_status, b->grid, b->stream);
        BatchSync sync;
        sync.nbr = b->nbr_ok && b->nbr_grid == b->grid ? b->d_nbr : nullptr;
        sync.done = b->d_done;
        sync.epoch = b->d_epoch;
        return launch_batch<TM>(b->d_probs, b->d_tiles, b->ntiles, n, b->d_level, b->d_bar, b->d_bar + 1,
                                b->d_status, sync, b->grid, b->npt, b->stream);
    };
    switch (b->prec) {
    case LBM_FP32_T64: return go(std::integral_constant<int, T_INT64>{});
    case LBM_FP32_TDF: return go(std::integral_constant<int, T_DF>{});
    case LBM_FP32_CONS: return go(std::integral_constant<int, T_CONS>{});
    default: return go(std::integral_constant<int, T_INT32>{});
    }
}
}  // namespace

extern "C" {

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    cudaFree(b->d_probs);
    cudaFree(b->d_tiles);
    cudaFree(b->d_nbr);
    cudaFree(b->d_done);
    cudaFree(b->d_epoch);
    cudaFree(b->d_segs);
    cudaFree(b->d_level);
    cudaFree(b->d_bar);
    cudaFree(b->d_status);
    cudaFreeHost(b->h_status);
    for (lbm_ctx* c : b->ctx) lbm_destroy(c);
    cudaGetLastError();
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

lbm_status lbm_batch_create(int nprob, const lbm_problem* probs, lbm_precision prec, void* stream,
                            lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_E_INVAL, "out must not be NULL");
    *out = nullptr;
    if (nprob < 1 || !probs) return bfail(nullptr, LBM_E_INVAL, "lbm_batch_create: need nprob >= 1 problems");
    if (prec != LBM_FP32 && prec != LBM_FP32_T64 && prec != LBM_FP32_TDF && prec != LBM_FP32_CONS)
        return bfail(nullptr, LBM_E_INVAL, "lbm_batch_create: the batch runs the FP32 modes only");
    lbm_batch* b = new lbm_batch();
    b->prec = prec;
    b->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&b->device);
    for (int p = 0; p < nprob; ++p) {
        const lbm_problem& q = probs[p];
        lbm_ctx* c = nullptr;
        lbm_status s = lbm_create(q.nx, q.ny, q.b, q.tau, q.dt, q.dx, &q.dvm, &q.diss, q.bc, prec, stream, &c);
        if (s != LBM_OK) {
            std::string m = "problem " + std::to_string(p) + ": " + g_create_err;
            lbm_batch_destroy(b);
            return bfail(nullptr, s, m);
        }
        b->ctx.push_back(c);
    }
    int tw = 0, th = 0;
    batch_tile_dims(&tw, &th);
    std::vector<int4> tiles;
    for (int p = 0; p < nprob; ++p)
        for (int y0 = 0; y0 < probs[p].ny; y0 += th)
            for (int x0 = 0; x0 < probs[p].nx; x0 += tw) tiles.push_back(make_int4(p, x0, y0, 0));
    b->ntiles = (int)tiles.size();
    b->tiles = tiles;
    for (int p = 0, base = 0; p < nprob; ++p) {
        const int tx = (probs[p].nx + tw - 1) / tw, ty = (probs[p].ny + th - 1) / th;
        b->tiles_x.push_back(tx);
        b->tiles_y.push_back(ty);
        b->tile_base.push_back(base);
        base += tx * ty;
        auto periodic = [&](int side) {
            return probs[p].bc[side].kind_lo == LBM_BC_PERIODIC || probs[p].bc[side].kind_hi == LBM_BC_PERIODIC;
        };
        b->periodic_x.push_back(periodic(LBM_SIDE_LEFT) || periodic(LBM_SIDE_RIGHT));
        b->periodic_y.push_back(periodic(LBM_SIDE_BOTTOM) || periodic(LBM_SIDE_TOP));
    }
    // temporal blocking: thin problems without periodic x sides
    b->tb_ok = true;
    for (int p = 0; p < nprob && b->tb_ok; ++p) {
        b->rows_max = probs[p].ny > b->rows_max ? probs[p].ny : b->rows_max;
        if (probs[p].ny > kBatchTbRowsMax) b->tb_ok = false;
        for (int side = LBM_SIDE_LEFT; side <= LBM_SIDE_RIGHT; ++side)
            if (probs[p].bc[side].kind_lo == LBM_BC_PERIODIC || probs[p].bc[side].kind_hi == LBM_BC_PERIODIC)
                b->tb_ok = false;
    }
    std::vector<int4> segs;
    if (b->tb_ok) {
        const int sw = batch_tb_width();
        for (int p = 0; p < nprob; ++p)
            for (int x0 = 0; x0 < probs[p].nx; x0 += sw) segs.push_back(make_int4(p, x0, 0, 0));
    }
    b->nsegs = (int)segs.size();
    std::vector<BatchProb> hp(nprob);
    int bbx = 0, bby = 0;
    batch_box_dims(&bbx, &bby);
    for (int p = 0; p < nprob; ++p) {
        hp[p].f[0] = static_cast<float*>(b->ctx[p]->f[0]);
        hp[p].f[1] = static_cast<float*>(b->ctx[p]->f[1]);
        hp[p].M = b->ctx[p]->mf;
        hp[p].G = b->ctx[p]->gf;
        // a problem that wraps in y inside its tile needs only its interior rows
        hp[p].wrap = batch_wraps_in_tile(hp[p].G) ? 1 : 0;
        const int rows = hp[p].wrap ? th : bby;
        hp[p].box_bytes = (unsigned)(sizeof(float) * 9 * bbx * rows);
        for (int k = 0; k < 2; ++k)
            if (!make_tmap_box(&hp[p].tm[k], b->ctx[p]->f[k], *b->ctx[p], bbx, rows)) {
                lbm_batch_destroy(b);
                return bfail(nullptr, LBM_E_CUDA, "lbm_batch_create: tensor maps unavailable on this driver");
            }
    }
    cudaError_t e = dev_malloc((void**)&b->d_probs, sizeof(BatchProb) * nprob);
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_tiles, sizeof(int4) * tiles.size());
    if (e == cudaSuccess && b->tb_ok) e = dev_malloc((void**)&b->d_segs, sizeof(int4) * segs.size());
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_level, sizeof(long long));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_probs, hp.data(), sizeof(BatchProb) * nprob, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && b->tb_ok)
        e = cudaMemcpyAsync(b->d_segs, segs.data(), sizeof(int4) * segs.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_level, 0, sizeof(long long), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        std::string m = std::string("lbm_batch_create: ") + cudaGetErrorString(e);
        lbm_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA, m);
    }
    for (int npt = 1; npt <= 2; ++npt)
        b->max_grid[npt] = prec == LBM_FP32_T64    ? batch_max_grid<T_INT64>(npt)
                           : prec == LBM_FP32_TDF  ? batch_max_grid<T_DF>(npt)
                           : prec == LBM_FP32_CONS ? batch_max_grid<T_CONS>(npt)
                                                   : batch_max_grid<T_INT32>(npt);
    b->nbr_cap = b->max_grid[1] > b->max_grid[2] ? b->max_grid[1] : b->max_grid[2];
    e = dev_malloc((void**)&b->d_nbr, sizeof(int) * (size_t)b->nbr_cap * kBatchMaxNbr);
    // one counter per CTA, and one more (index nbr_cap) that no CTA ever
    // publishes to (lbm_batch_plant_stall)
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_done, sizeof(unsigned long long) * (size_t)(b->nbr_cap + 1));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_epoch, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_done, 0, sizeof(unsigned long long) * (size_t)(b->nbr_cap + 1));
    if (e == cudaSuccess) e = cudaMemset(b->d_epoch, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        std::string m = std::string("lbm_batch_create: ") + cudaGetErrorString(e);
        lbm_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA, m);
    }
    b->npt = 1;
    b->grid = b->max_grid[1] < b->ntiles ? b->max_grid[1] : b->ntiles;
    if (b->tb_ok)
        for (int ns = 3; ns <= 7; ns += 2)
            b->tb_max_grid[ns] = prec == LBM_FP32_T64    ? batch_tb_max_grid<T_INT64>(ns, b->rows_max)
                                 : prec == LBM_FP32_TDF  ? batch_tb_max_grid<T_DF>(ns, b->rows_max)
                                 : prec == LBM_FP32_CONS ? batch_tb_max_grid<T_CONS>(ns, b->rows_max)
                                                         : batch_tb_max_grid<T_INT32>(ns, b->rows_max);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_init(lbm_batch* b, const void* const* rho, const void* const* ux, const void* const* uy,
                          const void* const* T) {
    if (!b || !rho || !ux || !uy || !T) return bfail(b, LBM_E_INVAL, "lbm_batch_init: NULL argument");
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        lbm_status s = lbm_init(b->ctx[p], rho[p], ux[p], uy[p], T[p]);
        if (s != LBM_OK) return bfail(b, s, "problem " + std::to_string(p) + ": " + b->ctx[p]->err);
    }
    cudaSetDevice(b->device);
    // the step counters and the grid barrier's words too: a launch that gave
    // up may have left the counters ahead of the epoch and the barrier with
    // arrivals that never completed
    if (cudaMemsetAsync(b->d_level, 0, sizeof(long long), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_done, 0, sizeof(unsigned long long) * (size_t)(b->nbr_cap + 1), b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->d_epoch, 0, sizeof(unsigned long long), b->stream) != cudaSuccess)
        return bfail(b, LBM_E_CUDA, "lbm_batch_init: clearing the batch state failed");
    b->step = 0;
    b->ready = true;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n) {
    NvtxRange nvtx_range("lbm_batch_step");
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    if (n < 0) return bfail(b, LBM_E_INVAL, "lbm_batch_step: n must be >= 0");
    if (!b->ready) return bfail(b, LBM_E_STATE, "lbm_batch_step before lbm_batch_init");
    if (n == 0) return LBM_OK;
    cudaSetDevice(b->device);
    cudaError_t e = batch_prepare_sync(b);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("lbm_batch_step: ") + cudaGetErrorString(e));
    // One graph (a single cooperative kernel node) per step count, captured on
    // a private stream and replayed there, ordered after and before the
    // caller's stream by events; replays read the level from device memory,
    // so one graph serves every call with the same n.
    if (b->graph_state >= 0 && b->graph_n != n) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        b->graph_n = -1;
        cudaStream_t keep = b->stream;
        b->stream = b->gstream;  // batch_launch queues on b->stream
        cudaGraph_t g = nullptr;
        cudaError_t be = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal);
        cudaError_t le = be == cudaSuccess ? batch_launch(b, n) : be;
        cudaError_t ce = be == cudaSuccess ? cudaStreamEndCapture(b->gstream, &g) : be;
        cudaError_t ie = (le == cudaSuccess && ce == cudaSuccess && g) ? cudaGraphInstantiate(&b->exec, g, 0) : le;
        b->stream = keep;
        if (le == cudaSuccess && ce == cudaSuccess && ie == cudaSuccess && g) {
            b->graph = g;
            b->graph_n = n;
            b->graph_state = 1;
        } else {
            if (g) cudaGraphDestroy(g);
            b->exec = nullptr;
            b->graph_state = -1;
            b->err = std::string("graph capture of the batch launch failed (") +
                     cudaGetErrorString(le != cudaSuccess ? le : (ce != cudaSuccess ? ce : ie)) +
                     "); launching directly";
        }
        cudaGetLastError();
    }
    if (b->exec && b->graph_n == n) {
        e = cudaEventRecord(b->ev_in, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->gstream, b->ev_in, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->gstream);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->gstream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
    } else {
        e = batch_launch(b, n);
    }
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("lbm_batch_step: ") + cudaGetErrorString(e));
    b->step += n;
    for (lbm_ctx* c : b->ctx) {
        c->step = b->step;
        c->cur = (int)(b->step & 1);
    }
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    cudaSetDevice(b->device);
    if (cudaMemcpyAsync(b->h_status, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, LBM_E_CUDA, "lbm_batch_sync: synchronising failed");
    if (*b->h_status & ST_TIMEOUT) return bfail(b, LBM_E_TIMEOUT, "a bounded wait between the batch kernel's CTAs gave up");
    if (*b->h_status & ST_NONPHYSICAL) return bfail(b, LBM_E_NONPHYSICAL, "a problem went non-physical");
    return LBM_OK;
}

lbm_ctx* lbm_batch_problem(lbm_batch* b, int p) {
    if (!b || p < 0 || p >= (int)b->ctx.size()) return nullptr;
    return b->ctx[(size_t)p];
}

lbm_status lbm_batch_info(const lbm_batch* b, int* grid, int* ntiles, int* graph) {
    if (!b) return LBM_E_INVAL;
    if (grid) *grid = b->grid;
    if (ntiles) *ntiles = b->ntiles;
    if (graph) *graph = b->graph_state;
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ von Neumann scan
namespace {

lbm_status vn_validate(const lbm_vn_case& q, int k) {
    if (!finite_pos(q.b) || !finite_pos(q.tau) || !finite_pos(q.dt) || !finite_pos(q.dx))
        return fail(nullptr, LBM_E_INVAL, "case %d: b, tau, dt, dx must be finite and > 0", k);
    if (!finite_pos(q.dvm.c1) || !finite_pos(q.dvm.c2) || !finite_pos(q.dvm.eta0) || q.dvm.c1 == q.dvm.c2)
        return fail(nullptr, LBM_E_INVAL, "case %d: c1, c2, eta0 must be finite, > 0, and c1 != c2", k);
    if (!(q.diss.beta >= 0.0 && q.diss.beta <= 0.5))
        return fail(nullptr, LBM_E_INVAL, "case %d: beta must lie in [0, 0.5]", k);
    for (int i = 0; i < 9; ++i)
        if (!(std::isfinite(q.diss.lambda[i]) && q.diss.lambda[i] >= 0.0))
            return fail(nullptr, LBM_E_INVAL, "case %d: lambda[%d] must be finite and >= 0", k, i);
    if (!finite_pos(q.state[0]) || !finite_pos(q.state[3]) || !std::isfinite(q.state[1]) ||
        !std::isfinite(q.state[2]))
        return fail(nullptr, LBM_E_INVAL, "case %d: the state needs rho > 0, T > 0, finite u", k);
    return LBM_OK;
}

struct StreamBuffers {  // device scratch of one call, released in stream order
    cudaStream_t st;
    std::vector<void*> ptrs;
    cudaError_t alloc(void** p, size_t bytes) {
        cudaError_t e = cudaMallocAsync(p, bytes, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~StreamBuffers() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

}  // namespace

extern "C" {

lbm_status lbm_vn_scan(const lbm_vn_case* cases, int ncases, const int* dirs, int ndirs, int nk,
                       double* radius, double* growth, void* stream) {
    NvtxRange nvtx_range("lbm_vn_scan");
    if (ncases < 0) return fail(nullptr, LBM_E_INVAL, "ncases must be >= 0");
    if (ncases == 0) return LBM_OK;
    if (!cases || !dirs) return fail(nullptr, LBM_E_INVAL, "cases and dirs must not be NULL");
    if (!radius && !growth) return fail(nullptr, LBM_E_INVAL, "radius and growth are both NULL");
    if (ndirs < 1 || ndirs > 64) return fail(nullptr, LBM_E_INVAL, "ndirs must lie in [1, 64]");
    if (nk < 1 || nk > 65536) return fail(nullptr, LBM_E_INVAL, "nk must lie in [1, 65536]");
    const long long total = (long long)ncases * ndirs * nk;
    if (total > (1LL << 31) - 1) return fail(nullptr, LBM_E_INVAL, "ncases * ndirs * nk exceeds 2^31 - 1");
    std::vector<int2> dv((size_t)ndirs);
    for (int d = 0; d < ndirs; ++d) {
        const int a = dirs[2 * d], b = dirs[2 * d + 1];
        if (a < -1024 || a > 1024 || b < -1024 || b > 1024 || (a == 0 && b == 0))
            return fail(nullptr, LBM_E_INVAL, "direction %d: components in [-1024, 1024], not both 0", d);
        dv[(size_t)d] = make_int2(a, b);
    }
    std::vector<VnCase> hv((size_t)ncases);
    for (int k = 0; k < ncases; ++k) {
        const lbm_vn_case& q = cases[k];
        const lbm_status s = vn_validate(q, k);
        if (s != LBM_OK) return s;
        hv[(size_t)k].M = build_model(q.b, q.tau, q.dt, q.dx, q.dvm, q.diss);
        hv[(size_t)k].rho = q.state[0];
        hv[(size_t)k].ux = q.state[1];
        hv[(size_t)k].uy = q.state[2];
        hv[(size_t)k].T = q.state[3];
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const bool r_dev = radius && is_device_ptr(radius), g_dev = growth && is_device_ptr(growth);
    StreamBuffers buf{st, {}};
    VnCase* d_cases = nullptr;
    int2* d_dirs = nullptr;
    double *d_J = nullptr, *d_r = r_dev ? radius : nullptr, *d_g = g_dev ? growth : nullptr;
    cudaError_t e = buf.alloc((void**)&d_cases, sizeof(VnCase) * hv.size());
    if (e == cudaSuccess) e = buf.alloc((void**)&d_dirs, sizeof(int2) * dv.size());
    if (e == cudaSuccess) e = buf.alloc((void**)&d_J, sizeof(double) * 81 * (size_t)ncases);
    if (e == cudaSuccess && !d_r) e = buf.alloc((void**)&d_r, sizeof(double) * (size_t)total);
    if (e == cudaSuccess && growth && !d_g) e = buf.alloc((void**)&d_g, sizeof(double) * (size_t)ncases);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lbm_vn_scan: allocating scratch");
    // pageable sources: each copy returns once its source has been staged
    e = cudaMemcpyAsync(d_cases, hv.data(), sizeof(VnCase) * hv.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_dirs, dv.data(), sizeof(int2) * dv.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_vn_scan(d_cases, ncases, d_dirs, ndirs, nk, d_J, d_r, d_g, st);
    if (e == cudaSuccess && radius && !r_dev)
        e = cudaMemcpyAsync(radius, d_r, sizeof(double) * (size_t)total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && growth && !g_dev)
        e = cudaMemcpyAsync(growth, d_g, sizeof(double) * (size_t)ncases, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ((radius && !r_dev) || (growth && !g_dev))) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lbm_vn_scan");
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------- batch launch shape
namespace {
void batch_drop_graph(lbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_n = -1;
    if (b->graph_state > 0) b->graph_state = 0;
}
}  // namespace

extern "C" {

lbm_status lbm_batch_set_launch(lbm_batch* b, const lbm_batch_launch* l) {
    if (!b || !l) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: NULL argument");
    int full = 0;
    if (l->block > 1) {
        if (l->block != 3 && l->block != 5 && l->block != 7)
            return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: block must be 0, 1, 3, 5 or 7");
        if (!b->tb_ok)
            return bfail(b, LBM_E_INVAL,
                         "lbm_batch_set_launch: temporal blocking needs problems of at most " +
                             std::to_string(kBatchTbRowsMax) + " rows and no periodic x sides");
        full = b->tb_max_grid[l->block] < b->nsegs ? b->tb_max_grid[l->block] : b->nsegs;
        if (full < 1) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: the blocking kernel does not fit");
    } else {
        if (l->block < 0) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: block must be 0, 1, 3, 5 or 7");
        if (l->npt != 1 && l->npt != 2) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: npt must be 1 or 2");
        full = b->max_grid[l->npt] < b->ntiles ? b->max_grid[l->npt] : b->ntiles;
    }
    if (l->grid < 0 || l->grid > full)
        return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: grid must lie in [0, " + std::to_string(full) + "]");
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->block = l->block > 1 ? l->block : 0;
    b->npt = l->block > 1 ? 1 : l->npt;
    b->grid = l->grid == 0 ? full : l->grid;
    batch_drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_inject_alloc_failure(long long after) {
    g_alloc_countdown.store(after < 0 ? -1 : after);
    return LBM_OK;
}

lbm_status lbm_batch_set_wait_limit(double seconds) {
    if (!(seconds > 0.0) || seconds > 60.0) return LBM_E_INVAL;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess ||
        khz <= 0) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    const long long cycles = (long long)(seconds * (double)khz * 1e3);
    if (batch_set_wait_cycles(cycles < 1 ? 1 : cycles) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    return LBM_OK;
}

lbm_status lbm_batch_plant_stall(lbm_batch* b, int cta) {
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    cudaSetDevice(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = batch_prepare_sync(b);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("lbm_batch_plant_stall: ") + cudaGetErrorString(e));
    if (cta < 0) {  // back to the lists of the current grid
        b->nbr_grid = -1;
        e = batch_prepare_sync(b);
        batch_drop_graph(b);
        return e == cudaSuccess ? LBM_OK : bfail(b, LBM_E_CUDA, "lbm_batch_plant_stall: restoring the lists failed");
    }
    if (b->block > 1 || !b->nbr_ok)
        return bfail(b, LBM_E_STATE, "lbm_batch_plant_stall: the current launch shape has no neighbour lists");
    if (cta >= b->grid)
        return bfail(b, LBM_E_INVAL, "lbm_batch_plant_stall: cta must lie in [0, " + std::to_string(b->grid) + ")");
    std::vector<int> lists;
    batch_neighbour_lists(b, b->grid, lists);
    int* row = lists.data() + (size_t)cta * kBatchMaxNbr;
    int j = 0;
    while (j < kBatchMaxNbr - 1 && row[j] >= 0) ++j;
    row[j] = b->nbr_cap;  // a counter no CTA publishes to
    e = cudaMemcpy(b->d_nbr, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice);
    batch_drop_graph(b);
    return e == cudaSuccess ? LBM_OK : bfail(b, LBM_E_CUDA, "lbm_batch_plant_stall: copying the lists failed");
}

lbm_status lbm_batch_get_launch(const lbm_batch* b, lbm_batch_launch* l) {
    if (!b || !l) return LBM_E_INVAL;
    l->npt = b->npt;
    l->grid = b->grid;
    l->block = b->block;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int steps, lbm_batch_launch* best, double* ms, int* n_candidates) {
    NvtxRange nvtx_range("lbm_batch_autotune");
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    if (steps < 1) return bfail(b, LBM_E_INVAL, "lbm_batch_autotune: steps must be >= 1");
    if (!b->ready) return bfail(b, LBM_E_STATE, "lbm_batch_autotune before lbm_batch_init");
    cudaSetDevice(b->device);
    // candidates: nodes per thread 1 or 2, a full wave or half of one
    lbm_batch_launch cand[8];
    int nc = 0;
    for (int npt = 1; npt <= 2; ++npt) {
        const int full = b->max_grid[npt] < b->ntiles ? b->max_grid[npt] : b->ntiles;
        cand[nc++] = {npt, full, 0};
        if (full >= 2) cand[nc++] = {npt, full / 2, 0};
    }
    if (b->tb_ok)
        for (int ns = 3; ns <= 7; ns += 2) {
            const int full = b->tb_max_grid[ns] < b->nsegs ? b->tb_max_grid[ns] : b->nsegs;
            if (full >= 1) cand[nc++] = {1, full, ns};
        }
    // save every problem's current level, the level counter and the status
    const int cur = (int)(b->step & 1);
    size_t total = 0;
    for (lbm_ctx* c : b->ctx) total += level_bytes(c);
    unsigned char* save = nullptr;
    long long* d_lsave = nullptr;
    unsigned* d_ssave = nullptr;
    cudaError_t e = dev_malloc((void**)&save, total);
    if (e == cudaSuccess) e = dev_malloc((void**)&d_lsave, sizeof(long long));
    if (e == cudaSuccess) e = dev_malloc((void**)&d_ssave, sizeof(unsigned));
    size_t off = 0;
    for (lbm_ctx* c : b->ctx) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(save + off, c->f[cur], level_bytes(c), cudaMemcpyDeviceToDevice, b->stream);
        off += level_bytes(c);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_lsave, b->d_level, sizeof(long long), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ssave, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->stream);
    auto restore = [&]() {
        cudaError_t r = cudaSuccess;
        size_t o = 0;
        for (lbm_ctx* c : b->ctx) {
            if (r == cudaSuccess)
                r = cudaMemcpyAsync(c->f[cur], save + o, level_bytes(c), cudaMemcpyDeviceToDevice, b->stream);
            o += level_bytes(c);
        }
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(b->d_level, d_lsave, sizeof(long long), cudaMemcpyDeviceToDevice, b->stream);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(b->d_status, d_ssave, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->stream);
        return r;
    };
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int keep_npt = b->npt, keep_grid = b->grid, keep_block = b->block;
    int bi = -1;
    float bms = 0.0f;
    for (int k = 0; k < nc && e == cudaSuccess; ++k) {
        b->npt = cand[k].npt;
        b->grid = cand[k].grid;
        b->block = cand[k].block;
        e = batch_prepare_sync(b);
        if (e == cudaSuccess) e = batch_launch(b, 1);  // untimed: first launch of the variant
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = batch_launch(b, steps);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float m = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m, t0, t1);
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess && ms) ms[k] = m / steps;
        if (e == cudaSuccess && (bi < 0 || m < bms)) {
            bi = k;
            bms = m;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(save);
    cudaFree(d_lsave);
    cudaFree(d_ssave);
    if (e != cudaSuccess || bi < 0) {
        b->npt = keep_npt;
        b->grid = keep_grid;
        b->block = keep_block;
        return bfail(b, LBM_E_CUDA, std::string("lbm_batch_autotune: ") + cudaGetErrorString(e));
    }
    b->npt = cand[bi].npt;
    b->grid = cand[bi].grid;
    b->block = cand[bi].block;
    batch_drop_graph(b);
    if (best) *best = cand[bi];
    if (n_candidates) *n_candidates = nc;
    return LBM_OK;
}

}  // extern "C"
