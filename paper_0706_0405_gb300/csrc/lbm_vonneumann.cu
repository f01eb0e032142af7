// lbm_vonneumann.cu -- batched linear stability analysis of the scheme
// (Sec. 3): for every case (a uniform state and the scheme's constants), wave
// direction and wave number, the spectral radius of the amplification matrix
// of Eqs. (SEC-VON-8, SEC-VON-12).
//
// Linearising the step of Eq. (SEC-VON-11) about a uniform state, a Fourier
// mode f_j(x) = F_j exp(i k.x) maps to G(k) F with
//     G(k) = diag(W_i(k)) + omega J,
//     W_i(k) = w_i0 + w_i1 e^{i kx dx} + w_i2 e^{-i kx dx} + w_i3 e^{i ky dx} + w_i4 e^{-i ky dx},
// where w_is are the folded five-point weights of the step (with -omega in
// w_i0) and J = d f^eq / d f is the Jacobian of the collision map at the
// state (Eqs. e4, e5, e7, e16-e18).  One thread builds and reduces one G(k).
#include "lbm_eig.cuh"
#include "lbm_launch.h"
#include "lbm_linear.cuh"

namespace lbm {

namespace {
constexpr int kVnThreads = 128;

inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

// Row i of J is g = (d f^eq_i / d q) (d q / d f) with q = (rho, ux, uy, T).
__global__ void __launch_bounds__(kVnThreads) k_vn_jacobian(const VnCase* __restrict__ cases, int ncases,
                                                            double* __restrict__ J) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncases) return;
    const VnCase C = cases[c];
    for (int i = 0; i < 9; ++i) {
        double a[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) a[k] = k == i ? 1.0 : 0.0;
        double h[4], g[9];
        feq_vjp(C.M, C.rho, C.ux, C.uy, C.T, a, h);
        moments_vjp(C.M, C.rho, C.ux, C.uy, C.T, h, g);
#pragma unroll
        for (int j = 0; j < 9; ++j) J[(size_t)c * 81 + i * 9 + j] = g[j];
    }
}

// radius[(c * ndirs + d) * nk + m] = max |eig G(k)| at k dx = pi m / (nk - 1)
// along direction dirs[d].
__global__ void __launch_bounds__(kVnThreads)
    k_vn_radius(const VnCase* __restrict__ cases, const double* __restrict__ J, const int2* __restrict__ dirs,
                int ncases, int ndirs, int nk, double* __restrict__ radius) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)ncases * ndirs * nk;
    if (t >= total) return;
    const int m = (int)(t % nk);
    const int d = (int)((t / nk) % ndirs);
    const int c = (int)(t / ((long long)nk * ndirs));
    const double frac = nk > 1 ? (double)m / (double)(nk - 1) : 0.0;  // k dx / pi
    double sx, cx, sy, cy;
    sincospi(dirs[d].x * frac, &sx, &cx);
    sincospi(dirs[d].y * frac, &sy, &cy);
    const Model<double>& M = cases[c].M;
    const double* Jc = J + (size_t)c * 81;
    cplx H[81];
    for (int i = 0; i < 9; ++i) {
        for (int j = 0; j < 9; ++j) H[i * 9 + j] = cplx{M.omega * Jc[i * 9 + j], 0.0};
        const double* w = M.w[i];
        H[i * 9 + i].re += w[0] + (w[1] + w[2]) * cx + (w[3] + w[4]) * cy;
        H[i * 9 + i].im += (w[1] - w[2]) * sx + (w[3] - w[4]) * sy;
    }
    hessenberg(H, 9);
    cplx ev[9];
    const int sweeps = hessenberg_eigenvalues(H, 9, ev);
    double r = 0.0;
    for (int k = 0; k < 9; ++k) r = fmax(r, cabs(ev[k]));
    radius[t] = sweeps < 0 ? NAN : r;
}

// growth[c] = max over the case's directions and wave numbers (NaN if any is NaN).
__global__ void k_vn_max(const double* __restrict__ radius, int ncases, int per, double* __restrict__ growth) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncases) return;
    double g = 0.0;
    for (int k = 0; k < per; ++k) {
        const double r = radius[(size_t)c * per + k];
        if (!(r <= g)) g = r;  // also keeps a NaN
        if (isnan(g)) break;
    }
    growth[c] = g;
}
}  // namespace

cudaError_t launch_vn_scan(const VnCase* cases, int ncases, const int2* dirs, int ndirs, int nk, double* J,
                           double* radius, double* growth, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    k_vn_jacobian<<<blocks_for(ncases, kVnThreads), kVnThreads, 0, st>>>(cases, ncases, J);
    const long long total = (long long)ncases * ndirs * nk;
    k_vn_radius<<<blocks_for(total, kVnThreads), kVnThreads, 0, st>>>(cases, J, dirs, ncases, ndirs, nk, radius);
    if (growth) k_vn_max<<<blocks_for(ncases, kVnThreads), kVnThreads, 0, st>>>(radius, ncases, ndirs * nk, growth);
    return cudaGetLastError();
}

}  // namespace lbm
