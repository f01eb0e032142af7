// lbm_eig.cuh -- eigenvalues of a small dense complex matrix in FP64, one
// matrix per thread: reduction to upper Hessenberg form by Givens rotations,
// then the shifted QR iteration on the Hessenberg matrix (Wilkinson shift
// from the trailing 2 x 2 block, deflation at negligible subdiagonal entries,
// ad hoc shifts after 10 and 20 stalled sweeps).  This is the textbook
// algorithm for the complex Schur form (Golub & Van Loan, Matrix
// Computations, Sec. 7.5), restricted to what the spectral radius needs: the
// rotations act only on the active diagonal block, since the eigenvalues do
// not depend on the blocks outside it.  Compiles for host and device.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

namespace lbm {

struct cplx {
    double re, im;
};

LBM_HD cplx cmake(double re, double im) { return cplx{re, im}; }
LBM_HD cplx cadd(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
LBM_HD cplx csub(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
LBM_HD cplx cmul(cplx a, cplx b) { return cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
LBM_HD cplx cconj(cplx a) { return cplx{a.re, -a.im}; }
LBM_HD cplx cscale(cplx a, double s) { return cplx{a.re * s, a.im * s}; }
LBM_HD double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
LBM_HD double cabs(cplx a) { return hypot(a.re, a.im); }
LBM_HD double cabs1(cplx a) { return fabs(a.re) + fabs(a.im); }

// a / b by scaling with the larger component of b (Smith's method).
LBM_HD cplx cdiv(cplx a, cplx b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return cplx{(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.re * r + b.im;
    return cplx{(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}

// Principal square root: sqrt(z) = sqrt((|z| + x) / 2) + i sgn(y) sqrt((|z| - x) / 2),
// with the smaller part formed as y / (2 * larger) to avoid cancellation.
LBM_HD cplx csqrt_p(cplx z) {
    if (z.re == 0.0 && z.im == 0.0) return cplx{0.0, 0.0};
    const double m = cabs(z);
    if (z.re >= 0.0) {
        const double t = sqrt(0.5 * (m + z.re));
        return cplx{t, z.im / (2.0 * t)};
    }
    const double t = sqrt(0.5 * (m - z.re));
    return cplx{fabs(z.im) / (2.0 * t), z.im >= 0.0 ? t : -t};
}

// Rotation G = [[c, s], [-conj(s), c]] (c real, c^2 + |s|^2 = 1) with
// G (x, y)^T = (r, 0)^T.
struct Givens {
    double c;
    cplx s;
};

LBM_HD Givens givens(cplx x, cplx y) {
    const double ay = cabs(y);
    if (ay == 0.0) return Givens{1.0, cplx{0.0, 0.0}};
    const double ax = cabs(x);
    if (ax == 0.0) return Givens{0.0, cconj(cscale(y, 1.0 / ay))};  // s = conj(y) / |y|
    const double r = hypot(ax, ay);
    const cplx ph = cscale(x, 1.0 / ax);                              // x / |x|
    return Givens{ax / r, cscale(cmul(ph, cconj(y)), 1.0 / r)};
}

// Rows p, p + 1 of H (n x n, row-major, leading dimension ld), columns
// c0 .. c1: (a, b) -> (c a + s b, -conj(s) a + c b).
LBM_HD void rot_rows(cplx* H, int ld, int p, int c0, int c1, Givens g) {
    for (int j = c0; j <= c1; ++j) {
        const cplx a = H[p * ld + j], b = H[(p + 1) * ld + j];
        H[p * ld + j] = cadd(cscale(a, g.c), cmul(g.s, b));
        H[(p + 1) * ld + j] = csub(cscale(b, g.c), cmul(cconj(g.s), a));
    }
}

// Columns p, p + 1 of H, rows r0 .. r1, multiplied from the right by G^H:
// (a, b) -> (c a + conj(s) b, -s a + c b).
LBM_HD void rot_cols(cplx* H, int ld, int p, int r0, int r1, Givens g) {
    for (int i = r0; i <= r1; ++i) {
        const cplx a = H[i * ld + p], b = H[i * ld + p + 1];
        H[i * ld + p] = cadd(cscale(a, g.c), cmul(cconj(g.s), b));
        H[i * ld + p + 1] = csub(cscale(b, g.c), cmul(g.s, a));
    }
}

// Reduce H (n x n) to upper Hessenberg form by unitary similarity.
LBM_HD void hessenberg(cplx* H, int n) {
    for (int k = 0; k + 2 < n; ++k)
        for (int j = n - 1; j >= k + 2; --j) {
            const Givens g = givens(H[(j - 1) * n + k], H[j * n + k]);
            rot_rows(H, n, j - 1, k, n - 1, g);
            H[j * n + k] = cplx{0.0, 0.0};
            rot_cols(H, n, j - 1, 0, n - 1, g);
        }
}

// Eigenvalues of the upper Hessenberg matrix H (destroyed) into ev[0..n).
// Returns the number of QR sweeps, or -1 if a block did not converge within
// kMaxSweeps sweeps (the unconverged eigenvalues are then NaN).
LBM_HD int hessenberg_eigenvalues(cplx* H, int n, cplx* ev) {
    constexpr int kMaxSweeps = 60;  // per eigenvalue
    constexpr double kEps = 2.220446049250313e-16;
    double anorm = 0.0;
    for (int k = 0; k < n * n; ++k) anorm = fmax(anorm, cabs1(H[k]));
    int hi = n - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            ev[0] = H[0];
            break;
        }
        // smallest l such that the block l..hi has no negligible subdiagonal
        int l = hi;
        while (l > 0) {
            double s = cabs1(H[(l - 1) * n + l - 1]) + cabs1(H[l * n + l]);
            if (s == 0.0) s = anorm;
            if (cabs1(H[l * n + l - 1]) <= kEps * s) {
                H[l * n + l - 1] = cplx{0.0, 0.0};
                break;
            }
            --l;
        }
        if (l == hi) {  // 1 x 1 block splits off
            ev[hi] = H[hi * n + hi];
            --hi;
            its = 0;
            continue;
        }
        if (its == kMaxSweeps) {
            for (int k = 0; k <= hi; ++k) ev[k] = cplx{NAN, NAN};
            return -1;
        }
        // shift
        cplx mu;
        const cplx a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
        const cplx c = H[hi * n + hi - 1], d = H[hi * n + hi];
        if (its == 10 || its == 20) {
            mu = cadd(d, cmake(fabs(c.re) + (hi >= 2 ? fabs(H[(hi - 1) * n + hi - 2].re) : 0.0), 0.0));
        } else {
            // eigenvalue of [[a, b], [c, d]] nearer to d: d - bc / (p + disc),
            // p = (a - d) / 2, disc = sqrt(p^2 + bc) signed to enlarge |p + disc|
            const cplx p = cscale(csub(a, d), 0.5);
            const cplx bc = cmul(b, c);
            cplx disc = csqrt_p(cadd(cmul(p, p), bc));
            if (p.re * disc.re + p.im * disc.im < 0.0) disc = cscale(disc, -1.0);
            const cplx den = cadd(p, disc);
            mu = (den.re == 0.0 && den.im == 0.0) ? d : csub(d, cdiv(bc, den));
        }
        // one explicit-shift QR sweep on the block l..hi: H - mu I = Q R, H <- R Q + mu I
        for (int k = l; k <= hi; ++k) H[k * n + k] = csub(H[k * n + k], mu);
        Givens gs[16];
        for (int k = l; k < hi; ++k) {
            gs[k - l] = givens(H[k * n + k], H[(k + 1) * n + k]);
            rot_rows(H, n, k, k, hi, gs[k - l]);
            H[(k + 1) * n + k] = cplx{0.0, 0.0};
        }
        for (int k = l; k < hi; ++k) rot_cols(H, n, k, l, (k + 2 <= hi ? k + 2 : hi), gs[k - l]);
        for (int k = l; k <= hi; ++k) H[k * n + k] = cadd(H[k * n + k], mu);
        ++its;
        ++total;
    }
    return total;
}

}  // namespace lbm
