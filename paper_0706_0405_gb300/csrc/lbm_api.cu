// lbm_api.cu -- the C ABI of liblbm (declared in include/lbm.h): context
// lifetime, parameter checks, derived constants, buffer management and the
// calls that queue the kernels on the caller's stream.  The batch calls are in
// lbm_api_batch.cu, the von Neumann scan in lbm_api_vn.cu.
#include "lbm_api_internal.h"

namespace lbm_api {
std::atomic<long long> g_alloc_countdown{-1};

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

// The device's address of page-locked host memory (cudaMallocHost,
// cudaHostRegister, torch pin_memory), or nullptr for any other pointer.  On
// a Grace-Blackwell node the GPU reads and writes such memory over the
// coherent CPU-GPU link, so a kernel can stream it directly instead of
// through a staging copy.
void* pinned_alias(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
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
        // C: the stencil's own centre weight; w[i][0] adds the identity and
        // the -omega of the relaxation
        double C = -4.0 * mu, E = mu, Wt = mu, N = mu, Sd = mu;
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
        M.w[i][0] = (1.0 - M.omega) + C;
        M.wi[i] = C;
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
    if (const void* alias = pinned_alias(p)) {  // read in place by the kernel
        *out = alias;
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
    // looked up once per process (a function-local static is initialised
    // once even when host threads race here)
    static const EncodeTiledFn fn = [] {
        EncodeTiledFn r = nullptr;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            r = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
        return r;
    }();
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

}  // namespace lbm_api

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

size_t lbm_level_bytes(int nx, int ny, lbm_precision prec) {
    if (nx < 1 || ny < 1 || nx > (1 << 24) || ny > (1 << 24) || prec < LBM_FP64 || prec > LBM_FP32_CONS) return 0;
    const size_t pitch = (size_t)((nx + 2 * PADX) + 31) / 32 * 32;
    return (size_t)(ny + 2) * 9 * pitch * (prec == LBM_FP64 ? 8 : 4);
}

lbm_status lbm_create(int nx, int ny, double b, double tau, double dt, double dx, const lbm_dvm* dvm,
                      const lbm_dissipation* diss, const lbm_bc bc[4], lbm_precision prec,
                      void* stream, void* f_buf0, void* f_buf1, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_E_INVAL, "out must not be NULL");
    *out = nullptr;
    lbm_status s = validate(nx, ny, b, tau, dt, dx, dvm, diss, bc, prec);
    if (s != LBM_OK) return s;
    const bool caller_f = f_buf0 || f_buf1;
    if (caller_f) {
        if (!f_buf0 || !f_buf1)
            return fail(nullptr, LBM_E_INVAL, "f_buf0 and f_buf1 must both be given or both be NULL");
        const size_t need = lbm_level_bytes(nx, ny, prec);
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(f_buf0), a1 = reinterpret_cast<uintptr_t>(f_buf1);
        if ((a0 | a1) % 256 != 0)
            return fail(nullptr, LBM_E_INVAL, "f_buf0 and f_buf1 must be 256-byte aligned");
        if ((a0 < a1 ? a1 - a0 : a0 - a1) < need)
            return fail(nullptr, LBM_E_INVAL, "f_buf0 and f_buf1 overlap (each needs %zu bytes)", need);
    }
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
    if (caller_f) {
        // the caller's buffers: device memory of this context's device
        void* bufs[2] = {f_buf0, f_buf1};
        for (int k = 0; k < 2; ++k) {
            cudaPointerAttributes at{};
            const bool dev_ok = cudaPointerGetAttributes(&at, bufs[k]) == cudaSuccess &&
                                (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
                                at.device == c->device;
            cudaGetLastError();
            if (!dev_ok) {
                delete c;
                return fail(nullptr, LBM_E_INVAL, "f_buf%d is not device memory of the current device", k);
            }
            c->f[k] = bufs[k];
        }
        c->f_owned = false;
    } else {
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = dev_malloc(&c->f[k], fbytes);
    }
    // status word, a spare, and the tile kernel's two scheduling counters
    if (e == cudaSuccess) e = dev_malloc((void**)&c->d_status, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_status, sizeof(unsigned));
    const int np = c->prec == LBM_FP64 ? conservation_partials(c->gd) : conservation_partials(c->gf);
    if (e == cudaSuccess) e = dev_malloc((void**)&c->d_partials, sizeof(double) * 4 * np);
    if (e == cudaSuccess) e = dev_malloc((void**)&c->d_sums, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_sums, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[0], 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[1], 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 4 * sizeof(unsigned), c->stream);
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
    if (c->f_owned) {  // caller-owned level buffers are never freed here
        cudaFree(c->f[0]);
        cudaFree(c->f[1]);
    }
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
    bool host_any = false, stage_any = false;
    for (int k = 0; k < 4; ++k) {
        dev[k] = nullptr;
        if (!out[k]) continue;
        if (is_device_ptr(out[k])) {
            dev[k] = out[k];
            continue;
        }
        host_any = true;
        dev[k] = pinned_alias(out[k]);  // page-locked: the kernel writes it in place
        if (!dev[k]) stage_any = true;
    }
    if (stage_any && (s = ensure_stage(c, 9 * fb)) != LBM_OK) return s;
    void* aliased[4];
    for (int k = 0; k < 4; ++k) {
        aliased[k] = dev[k];
        if (out[k] && !dev[k]) dev[k] = static_cast<char*>(c->d_stage) + k * fb;
    }
    cudaError_t e = dispatch(c, [&](auto tag, auto tm) {
        using S = decltype(tag);
        constexpr int TM = decltype(tm)::value;
        return launch_moments<S, TM>(static_cast<const S*>(c->f[c->cur]), (S*)dev[0], (S*)dev[1], (S*)dev[2],
                                     (S*)dev[3], model_of<S>(c), grid_of<S>(c), c->d_status, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_moments");
    for (int k = 0; k < 4; ++k)
        if (out[k] && !aliased[k])
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

extern "C" lbm_status lbm_inject_alloc_failure(long long after) {
    g_alloc_countdown.store(after < 0 ? -1 : after);
    return LBM_OK;
}
