// lbm_api_vn.cu -- lbm_vn_scan of the C ABI (include/lbm.h): the batched
// von Neumann scan's argument checks, case set-up and launch.
#include "lbm_api_internal.h"

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
