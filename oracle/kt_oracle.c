/*
 * kt_oracle.c -- plain serial FP64 restatement of the Kataoka-Tsutahara D2V9
 * finite-difference lattice Boltzmann step with the added dissipation term of
 * Pan, Xu, Zhang & Jiang, "Lattice Boltzmann Approach to High-Speed
 * Compressible Flows" (IJMPC 2007).
 *
 * TEST INFRASTRUCTURE.  This file is the oracle the CUDA path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant with the CUDA
 * library; the two are written independently from the paper.
 *
 * It follows the paper's algorithm in the paper's order, one node at a time:
 *   (i)   ghost cells from the boundary kinds            (Sec. 4, Eq. Riemann-3 text)
 *   (ii)  moments rho, u, T                               (Eqs. e4, e5, e7)
 *   (iii) equilibrium f^eq                                (Eqs. e16, e17, e18)
 *   (iv)  beta-upwind first derivatives per axis          (Eqs. SEC-VON-2a, 2b)
 *         and central second derivatives                  (text after SEC-VON-11)
 *   (v)   forward-Euler update with BGK relaxation and
 *         the dissipation term                            (Eq. SEC-VON-11)
 *
 * Readings of the paper taken here (each is pinned by a test):
 *   - Eq. (e14): the diagonal velocities are c2 (cos th, sin th), |v| = c2; the
 *     printed (cos, cos) duplicates two velocities and breaks Eqs. (e4)-(e8).
 *   - Eq. (e17): A_0 = (b - 2) T / eta0^2; the printed eta0^1 breaks the mass and
 *     energy identities.
 *   - Eq. (SEC-VON-1): the collision factor per step is omega = dt / tau, the
 *     paper's 1/tau with dt equal to the Knudsen number.
 *   - R = 1 (non-dimensional), so P = rho T.
 *   - Boundary mechanics (the paper only names the kinds): one ghost layer;
 *     periodic = wrap, outflow = copy of the adjacent interior node,
 *     Dirichlet = f^eq of the prescribed state, reflecting = the adjacent
 *     interior node with the wall-normal velocity component mirrored.
 *     A side may switch kind/state at an along-side coordinate s0 + s1 * t,
 *     which expresses the double-Mach-reflection wall start and the moving
 *     exact shock position on the top boundary.
 *   - Cell-centred nodes: x_j = (j + 1/2) dx, y_k = (k + 1/2) dx (dx = dy).
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared [-fopenmp].  FMA contraction
 * is disabled so that the result is the same on every host architecture.
 * Nodes are independent within a step, so the optional OpenMP node loop does
 * not change any result.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { KT_PERIODIC = 0, KT_OUTFLOW = 1, KT_DIRICHLET = 2, KT_REFLECT = 3 };
enum { KT_LEFT = 0, KT_RIGHT = 1, KT_BOTTOM = 2, KT_TOP = 3 };

typedef struct {
    int kind_lo;          /* kind where the along-side coordinate < s0 + s1 t */
    int kind_hi;          /* kind elsewhere */
    double split0;        /* s0 */
    double split_speed;   /* s1 */
    double state_lo[4];   /* (rho, ux, uy, T) of a Dirichlet part below the split */
    double state_hi[4];   /* ... above the split */
} kt_side;

typedef struct {
    int nx, ny;
    double b;             /* b = 2 / (gamma - 1), Eq. (e2) text */
    double tau, dt, dx;   /* relaxation time, time step, grid step (dx = dy) */
    double c1, c2, eta0;  /* DVM constants, Eqs. (e14), (e15) */
    double beta;          /* upwind blend, Eqs. (SEC-VON-2a/2b), 0 <= beta <= 1/2 */
    double lambda[9];     /* dissipation coefficients, Eq. (SEC-VON-11) */
    kt_side side[4];      /* left (x=0), right, bottom (y=0), top */
} kt_config;

/* Direction signs of the nine velocities of Eq. (e14):
 * i = 1..4 are c1 (cos(pi (i+1)/2), sin(pi (i+1)/2)),
 * i = 5..8 are c2 (cos(pi ((i+1)/2 + 1/4)), sin(same)).
 * Kept as integers so that the upwind choice of Eqs. (SEC-VON-2a/2b) never
 * depends on the round-off of cos(pi/2). */
static const int SX[9] = {0, -1, 0, 1, 0, -1, 1, 1, -1};
static const int SY[9] = {0, 0, -1, 0, 1, -1, -1, 1, 1};

static int omp_threads = 1;

void kt_set_threads(int n) { omp_threads = n < 1 ? 1 : n; }

int kt_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* Eq. (e14): the velocity table. */
void kt_velocities(double c1, double c2, double vx[9], double vy[9]) {
    double diag = c2 / sqrt(2.0);
    for (int i = 0; i < 9; ++i) {
        double mag = (i == 0) ? 0.0 : (i <= 4 ? c1 : diag);
        vx[i] = SX[i] * mag;
        vy[i] = SY[i] * mag;
    }
}

/* Eq. (e15): eta_i. */
static double eta_of(const kt_config* c, int i) { return i == 0 ? c->eta0 : 0.0; }

/* Mirror map of a reflecting wall: the population whose velocity has the
 * wall-normal component reversed and the tangential one kept. */
static int mirror(int i, int normal_is_x) {
    for (int j = 0; j < 9; ++j) {
        int same_group = (i == 0 && j == 0) || (i >= 1 && i <= 4 && j >= 1 && j <= 4) ||
                         (i >= 5 && j >= 5);
        if (!same_group) continue;
        if (normal_is_x && SX[j] == -SX[i] && SY[j] == SY[i]) return j;
        if (!normal_is_x && SY[j] == -SY[i] && SX[j] == SX[i]) return j;
    }
    return -1;
}

/* Eqs. (e16)-(e18): f_i^eq = rho (A_i + B_i v_i.u + D_i (v_i.u)^2). */
void kt_feq(const kt_config* c, double rho, double ux, double uy, double T, double feq[9]) {
    double b = c->b, c1s = c->c1 * c->c1, c2s = c->c2 * c->c2, e0s = c->eta0 * c->eta0;
    double u2 = ux * ux + uy * uy;
    double vx[9], vy[9];
    kt_velocities(c->c1, c->c2, vx, vy);

    double A0 = (b - 2.0) * T / e0s;
    double A1 = (-c2s + ((b - 2.0) * c2s / e0s + 2.0) * T + c2s / c1s * u2) / (4.0 * (c1s - c2s));
    double A5 = (-c1s + ((b - 2.0) * c1s / e0s + 2.0) * T + c1s / c2s * u2) / (4.0 * (c2s - c1s));
    double B1 = (-c2s + (b + 2.0) * T + u2) / (2.0 * c1s * (c1s - c2s));
    double B5 = (-c1s + (b + 2.0) * T + u2) / (2.0 * c2s * (c2s - c1s));
    double D1 = 1.0 / (2.0 * c1s * c1s);
    double D5 = 1.0 / (2.0 * c2s * c2s);

    feq[0] = rho * A0;
    for (int i = 1; i < 9; ++i) {
        double vu = vx[i] * ux + vy[i] * uy;
        if (i <= 4)
            feq[i] = rho * (A1 + B1 * vu + D1 * vu * vu);
        else
            feq[i] = rho * (A5 + B5 * vu + D5 * vu * vu);
    }
}

/* Eqs. (e4), (e5), (e7): rho = sum f, rho u = sum f v,
 * rho (b T + u^2) = sum f (v^2 + eta^2); out = (rho, ux, uy, T). */
void kt_moments(const kt_config* c, const double f[9], double out[4]) {
    double vx[9], vy[9];
    kt_velocities(c->c1, c->c2, vx, vy);
    double rho = 0.0, jx = 0.0, jy = 0.0, E = 0.0;
    for (int i = 0; i < 9; ++i) {
        double eta = eta_of(c, i);
        rho += f[i];
        jx += f[i] * vx[i];
        jy += f[i] * vy[i];
        E += f[i] * (vx[i] * vx[i] + vy[i] * vy[i] + eta * eta);
    }
    double ux = jx / rho, uy = jy / rho;
    out[0] = rho;
    out[1] = ux;
    out[2] = uy;
    out[3] = (E / rho - (ux * ux + uy * uy)) / c->b;
}

/* Storage: f[i][k][j], k = 0..ny+1, j = 0..nx+1; k = 0, ny+1 and j = 0, nx+1
 * are the ghost layer.  Interior node (jj, kk) (0-based) sits at (jj+1, kk+1). */
static size_t at(const kt_config* c, int i, int k, int j) {
    return ((size_t)i * (size_t)(c->ny + 2) + (size_t)k) * (size_t)(c->nx + 2) + (size_t)j;
}

size_t kt_field_len(const kt_config* c) { return (size_t)9 * (c->ny + 2) * (c->nx + 2); }

/* Value of population i in the ghost cell of `side` next to interior cell
 * (k, j) (storage indices); `along` is the ghost cell's centre coordinate along
 * the side and t the time of the level being filled. */
static double ghost_value(const kt_config* c, const double* f, int side, int i, int k, int j,
                          double along, double t) {
    const kt_side* s = &c->side[side];
    double split = s->split0 + s->split_speed * t;
    int lo = along < split;
    int kind = lo ? s->kind_lo : s->kind_hi;
    const double* st = lo ? s->state_lo : s->state_hi;
    switch (kind) {
    case KT_PERIODIC:
        if (side == KT_LEFT) return f[at(c, i, k, c->nx)];
        if (side == KT_RIGHT) return f[at(c, i, k, 1)];
        if (side == KT_BOTTOM) return f[at(c, i, c->ny, j)];
        return f[at(c, i, 1, j)];
    case KT_OUTFLOW:
        return f[at(c, i, k, j)];
    case KT_DIRICHLET: {
        double feq[9];
        kt_feq(c, st[0], st[1], st[2], st[3], feq);
        return feq[i];
    }
    case KT_REFLECT:
        return f[at(c, mirror(i, side == KT_LEFT || side == KT_RIGHT), k, j)];
    }
    return NAN;
}

/* Step (i): fill the ghost layer of f for time t.  Corner ghosts are never read
 * by the five-point stencil and are set to NaN so that a stray read shows. */
void kt_fill_ghosts(const kt_config* c, double* f, double t) {
    int nx = c->nx, ny = c->ny;
    for (int i = 0; i < 9; ++i) {
        f[at(c, i, 0, 0)] = NAN;
        f[at(c, i, 0, nx + 1)] = NAN;
        f[at(c, i, ny + 1, 0)] = NAN;
        f[at(c, i, ny + 1, nx + 1)] = NAN;
    }
    for (int k = 1; k <= ny; ++k) {
        double y = ((double)(k - 1) + 0.5) * c->dx;
        for (int i = 0; i < 9; ++i) {
            f[at(c, i, k, 0)] = ghost_value(c, f, KT_LEFT, i, k, 1, y, t);
            f[at(c, i, k, nx + 1)] = ghost_value(c, f, KT_RIGHT, i, k, nx, y, t);
        }
    }
    for (int j = 1; j <= nx; ++j) {
        double x = ((double)(j - 1) + 0.5) * c->dx;
        for (int i = 0; i < 9; ++i) {
            f[at(c, i, 0, j)] = ghost_value(c, f, KT_BOTTOM, i, 1, j, x, t);
            f[at(c, i, ny + 1, j)] = ghost_value(c, f, KT_TOP, i, ny, j, x, t);
        }
    }
}

/* Steps (ii)-(v) at one interior node (k, j) (storage indices), reading level n
 * from f (ghosts filled) and writing the nine level-(n+1) values to out. */
static void node_update(const kt_config* c, const double* f, int k, int j, double out[9]) {
    double vx[9], vy[9], fc[9], m[4], feq[9];
    kt_velocities(c->c1, c->c2, vx, vy);
    for (int i = 0; i < 9; ++i) fc[i] = f[at(c, i, k, j)];

    kt_moments(c, fc, m);                      /* Eqs. (e4), (e5), (e7) */
    kt_feq(c, m[0], m[1], m[2], m[3], feq);    /* Eqs. (e16)-(e18) */

    double beta = c->beta, dx = c->dx, dt = c->dt;
    for (int i = 0; i < 9; ++i) {
        double f0 = fc[i];
        double fE = f[at(c, i, k, j + 1)], fW = f[at(c, i, k, j - 1)];
        double fN = f[at(c, i, k + 1, j)], fS = f[at(c, i, k - 1, j)];
        double dfx, dfy;
        /* Eqs. (SEC-VON-2a) (v >= 0) and (SEC-VON-2b) (v < 0), per axis. */
        if (SX[i] >= 0)
            dfx = (beta * fE + (1.0 - 2.0 * beta) * f0 - (1.0 - beta) * fW) / dx;
        else
            dfx = ((1.0 - beta) * fE - (1.0 - 2.0 * beta) * f0 - beta * fW) / dx;
        if (SY[i] >= 0)
            dfy = (beta * fN + (1.0 - 2.0 * beta) * f0 - (1.0 - beta) * fS) / dx;
        else
            dfy = ((1.0 - beta) * fN - (1.0 - 2.0 * beta) * f0 - beta * fS) / dx;
        /* Central second differences for the dissipation term. */
        double lap = (fE - 2.0 * f0 + fW) / (dx * dx) + (fN - 2.0 * f0 + fS) / (dx * dx);
        /* Eq. (SEC-VON-11) solved for f(t + dt), collision factor dt / tau. */
        out[i] = f0 - (vx[i] * dfx + vy[i] * dfy) * dt + c->lambda[i] * lap * dt +
                 (dt / c->tau) * (feq[i] - f0);
    }
}

static int nonphysical(const kt_config* c, const double v[9]) {
    double m[4];
    kt_moments(c, v, m);
    return !(m[0] > 0.0) || !(m[3] > 0.0) || !isfinite(m[1]) || !isfinite(m[2]);
}

/* Initial condition: f = f^eq of the given fields (row-major ny x nx arrays);
 * the ghost layer is left as NaN until the first step fills it. */
void kt_init(const kt_config* c, const double* rho, const double* ux, const double* uy,
             const double* T, double* f) {
    size_t len = kt_field_len(c);
    for (size_t q = 0; q < len; ++q) f[q] = NAN;
    for (int kk = 0; kk < c->ny; ++kk)
        for (int jj = 0; jj < c->nx; ++jj) {
            size_t p = (size_t)kk * c->nx + jj;
            double feq[9];
            kt_feq(c, rho[p], ux[p], uy[p], T[p], feq);
            for (int i = 0; i < 9; ++i) f[at(c, i, kk + 1, jj + 1)] = feq[i];
        }
}

/* Advance nsteps steps starting at step index n0 (time n0 dt).  f holds the
 * state and receives the result; work is scratch of the same length.
 * Returns the number of nodes of the final level with rho <= 0, T <= 0 or a
 * non-finite velocity. */
long kt_run(const kt_config* c, double* f, double* work, long nsteps, long n0) {
    double* a = f;
    double* bnew = work;
    for (long s = 0; s < nsteps; ++s) {
        double t = (double)(n0 + s) * c->dt;
        kt_fill_ghosts(c, a, t);
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(omp_threads)
#endif
        for (int k = 1; k <= c->ny; ++k) {
            for (int j = 1; j <= c->nx; ++j) {
                double out[9];
                node_update(c, a, k, j, out);
                for (int i = 0; i < 9; ++i) bnew[at(c, i, k, j)] = out[i];
            }
        }
        double* tmp = a;
        a = bnew;
        bnew = tmp;
    }
    if (a != f) memcpy(f, a, kt_field_len(c) * sizeof(double));
    long bad = 0;
    for (int k = 1; k <= c->ny; ++k)
        for (int j = 1; j <= c->nx; ++j) {
            double v[9];
            for (int i = 0; i < 9; ++i) v[i] = f[at(c, i, k, j)];
            bad += nonphysical(c, v);
        }
    return bad;
}

/* The same steps with the state held in FP32 between steps, the arithmetic
 * still FP64: after each ghost fill and each update, every stored value is
 * rounded to the nearest FP32 number.  Not from the paper: this is the floor
 * that an FP32 state (the storage of the library's FP32 modes) puts under
 * the error of any implementation that stores f in FP32, whatever precision
 * its arithmetic has. */
static void round_to_f32(double* v, size_t len) {
    for (size_t q = 0; q < len; ++q) v[q] = (double)(float)v[q];
}

long kt_run_f32_storage(const kt_config* c, double* f, double* work, long nsteps, long n0) {
    const size_t len = kt_field_len(c);
    double* a = f;
    double* bnew = work;
    round_to_f32(a, len);
    for (long s = 0; s < nsteps; ++s) {
        double t = (double)(n0 + s) * c->dt;
        kt_fill_ghosts(c, a, t);
        round_to_f32(a, len);
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(omp_threads)
#endif
        for (int k = 1; k <= c->ny; ++k) {
            for (int j = 1; j <= c->nx; ++j) {
                double out[9];
                node_update(c, a, k, j, out);
                for (int i = 0; i < 9; ++i) bnew[at(c, i, k, j)] = (double)(float)out[i];
            }
        }
        double* tmp = a;
        a = bnew;
        bnew = tmp;
    }
    if (a != f) memcpy(f, a, len * sizeof(double));
    long bad = 0;
    for (int k = 1; k <= c->ny; ++k)
        for (int j = 1; j <= c->nx; ++j) {
            double v[9];
            for (int i = 0; i < 9; ++i) v[i] = f[at(c, i, k, j)];
            bad += nonphysical(c, v);
        }
    return bad;
}

/* One step evaluated only at the listed interior nodes (node = kk * nx + jj),
 * from the level-n state f at step index n.  f's ghost layer is (re)filled
 * for time n dt.  out receives count x 9 values. */
void kt_step_nodes(const kt_config* c, double* f, long n, const long* nodes, long count,
                   double* out) {
    kt_fill_ghosts(c, f, (double)n * c->dt);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(omp_threads)
#endif
    for (long q = 0; q < count; ++q) {
        int kk = (int)(nodes[q] / c->nx), jj = (int)(nodes[q] % c->nx);
        node_update(c, f, kk + 1, jj + 1, out + 9 * q);
    }
}

/* Macroscopic fields (rho, ux, uy, T) of the interior, row-major ny x nx. */
void kt_fields(const kt_config* c, const double* f, double* rho, double* ux, double* uy,
               double* T) {
    for (int kk = 0; kk < c->ny; ++kk)
        for (int jj = 0; jj < c->nx; ++jj) {
            double v[9], m[4];
            for (int i = 0; i < 9; ++i) v[i] = f[at(c, i, kk + 1, jj + 1)];
            kt_moments(c, v, m);
            size_t p = (size_t)kk * c->nx + jj;
            rho[p] = m[0];
            ux[p] = m[1];
            uy[p] = m[2];
            T[p] = m[3];
        }
}

/* Conserved totals over the interior: sum rho, sum rho ux, sum rho uy,
 * sum rho (b T + u^2), each the plain sum of Eqs. (e4), (e5), (e7). */
void kt_sums(const kt_config* c, const double* f, double out[4]) {
    double vx[9], vy[9];
    kt_velocities(c->c1, c->c2, vx, vy);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int kk = 0; kk < c->ny; ++kk)
        for (int jj = 0; jj < c->nx; ++jj)
            for (int i = 0; i < 9; ++i) {
                double v = f[at(c, i, kk + 1, jj + 1)];
                double eta = eta_of(c, i);
                s[0] += v;
                s[1] += v * vx[i];
                s[2] += v * vy[i];
                s[3] += v * (vx[i] * vx[i] + vy[i] * vy[i] + eta * eta);
            }
    for (int q = 0; q < 4; ++q) out[q] = s[q];
}

/* ------------------------------------------------------------------------
 * Adjoint (transpose of the linearised step).  Written from the same
 * equations: the step is out_i(x) = sum over the star of coefficients times
 * f_i(x + s), plus (dt / tau) f^eq_i(moments f(x)); its transpose scatters
 * each coefficient times the adjoint of out_i(x) back to f_i(x + s) (through
 * the ghost rule when x + s is a ghost cell) and adds
 * (dt / tau) sum_i abar_i J_ij with J = d f^eq / d f at f(x).
 * ---------------------------------------------------------------------- */

/* d out_i(x) / d f_i(x + s) of Eqs. (SEC-VON-2a/2b, SEC-VON-11) for the star
 * s = centre, +x, -x, +y, -y, without the f^eq term. */
static void star_coeffs(const kt_config* c, int i, double coef[5]) {
    double vx[9], vy[9];
    kt_velocities(c->c1, c->c2, vx, vy);
    double beta = c->beta, dt = c->dt, dx = c->dx, lam = c->lambda[i] * dt / (dx * dx);
    double ax = vx[i] * dt / dx, ay = vy[i] * dt / dx;
    double cE, cC, cW, cN, cS;
    if (SX[i] >= 0) { /* -ax (beta fE + (1 - 2 beta) f0 - (1 - beta) fW) */
        cE = -ax * beta;
        cC = -ax * (1.0 - 2.0 * beta);
        cW = ax * (1.0 - beta);
    } else { /* -ax ((1 - beta) fE - (1 - 2 beta) f0 - beta fW) */
        cE = -ax * (1.0 - beta);
        cC = ax * (1.0 - 2.0 * beta);
        cW = ax * beta;
    }
    if (SY[i] >= 0) {
        cN = -ay * beta;
        cC += -ay * (1.0 - 2.0 * beta);
        cS = ay * (1.0 - beta);
    } else {
        cN = -ay * (1.0 - beta);
        cC += ay * (1.0 - 2.0 * beta);
        cS = ay * beta;
    }
    coef[0] = 1.0 + cC - 4.0 * lam - dt / c->tau;
    coef[1] = cE + lam;
    coef[2] = cW + lam;
    coef[3] = cN + lam;
    coef[4] = cS + lam;
}

/* Derivatives of f^eq_i (Eqs. e16-e18) with respect to q = (rho, ux, uy, T):
 * dF[i][m]. */
static void feq_dq(const kt_config* c, double rho, double ux, double uy, double T, double dF[9][4]) {
    double b = c->b, c1s = c->c1 * c->c1, c2s = c->c2 * c->c2, e0s = c->eta0 * c->eta0;
    double u2 = ux * ux + uy * uy;
    double vx[9], vy[9];
    kt_velocities(c->c1, c->c2, vx, vy);
    /* A, B as written in Eqs. (e17), (e18) and their partial derivatives in T
     * and in u^2. */
    double q1 = 4.0 * (c1s - c2s), q5 = 4.0 * (c2s - c1s);
    double A1 = (-c2s + ((b - 2.0) * c2s / e0s + 2.0) * T + c2s / c1s * u2) / q1;
    double A5 = (-c1s + ((b - 2.0) * c1s / e0s + 2.0) * T + c1s / c2s * u2) / q5;
    double A1T = ((b - 2.0) * c2s / e0s + 2.0) / q1, A1u = (c2s / c1s) / q1;
    double A5T = ((b - 2.0) * c1s / e0s + 2.0) / q5, A5u = (c1s / c2s) / q5;
    double d1 = 2.0 * c1s * (c1s - c2s), d5 = 2.0 * c2s * (c2s - c1s);
    double B1 = (-c2s + (b + 2.0) * T + u2) / d1, B5 = (-c1s + (b + 2.0) * T + u2) / d5;
    double B1T = (b + 2.0) / d1, B1u = 1.0 / d1, B5T = (b + 2.0) / d5, B5u = 1.0 / d5;
    double D1 = 1.0 / (2.0 * c1s * c1s), D5 = 1.0 / (2.0 * c2s * c2s);
    /* i = 0: F = rho (b - 2) T / eta0^2 */
    dF[0][0] = (b - 2.0) * T / e0s;
    dF[0][1] = 0.0;
    dF[0][2] = 0.0;
    dF[0][3] = rho * (b - 2.0) / e0s;
    for (int i = 1; i < 9; ++i) {
        double A = i <= 4 ? A1 : A5, AT = i <= 4 ? A1T : A5T, Au = i <= 4 ? A1u : A5u;
        double B = i <= 4 ? B1 : B5, BT = i <= 4 ? B1T : B5T, Bu = i <= 4 ? B1u : B5u;
        double D = i <= 4 ? D1 : D5;
        double vu = vx[i] * ux + vy[i] * uy;
        dF[i][0] = A + B * vu + D * vu * vu;
        /* d/dux: A and B through u^2 (d u^2 / d ux = 2 ux), and v.u */
        dF[i][1] = rho * (Au * 2.0 * ux + Bu * 2.0 * ux * vu + B * vx[i] + 2.0 * D * vu * vx[i]);
        dF[i][2] = rho * (Au * 2.0 * uy + Bu * 2.0 * uy * vu + B * vy[i] + 2.0 * D * vu * vy[i]);
        dF[i][3] = rho * (AT + BT * vu);
    }
}

/* Derivatives of q = (rho, ux, uy, T) (Eqs. e4, e5, e7) with respect to f_j
 * at the populations f: dq[m][j]. */
static void moments_df(const kt_config* c, const double f[9], double dq[4][9]) {
    double m[4], vx[9], vy[9];
    kt_moments(c, f, m);
    kt_velocities(c->c1, c->c2, vx, vy);
    double rho = m[0], ux = m[1], uy = m[2], T = m[3];
    for (int j = 0; j < 9; ++j) {
        double eta = eta_of(c, j);
        double dx = vx[j] - ux, dy = vy[j] - uy;
        dq[0][j] = 1.0;
        dq[1][j] = dx / rho;
        dq[2][j] = dy / rho;
        /* T = (E / rho - u.u) / b, E = sum f (v^2 + eta^2) */
        dq[3][j] = (dx * dx + dy * dy + eta * eta - c->b * T) / (c->b * rho);
    }
}

/* Jacobian J[i][j] = d f^eq_i / d f_j at the populations f. */
void kt_feq_jacobian(const kt_config* c, const double f[9], double J[81]) {
    double m[4], dF[9][4], dq[4][9];
    kt_moments(c, f, m);
    feq_dq(c, m[0], m[1], m[2], m[3], dF);
    moments_df(c, f, dq);
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) s += dF[i][q] * dq[q][j];
            J[i * 9 + j] = s;
        }
}

/* Vector-Jacobian products: qbar_m = sum_i abar_i dF_i/dq_m at the state q,
 * and abar_j = sum_m qbar_m dq_m/df_j at the populations f. */
void kt_feq_vjp(const kt_config* c, const double q[4], const double abar[9], double qbar[4]) {
    double dF[9][4];
    feq_dq(c, q[0], q[1], q[2], q[3], dF);
    for (int m = 0; m < 4; ++m) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += abar[i] * dF[i][m];
        qbar[m] = s;
    }
}

void kt_moments_vjp(const kt_config* c, const double f[9], const double qbar[4], double abar[9]) {
    double dq[4][9];
    moments_df(c, f, dq);
    for (int j = 0; j < 9; ++j) {
        double s = 0.0;
        for (int m = 0; m < 4; ++m) s += qbar[m] * dq[m][j];
        abar[j] = s;
    }
}

/* Route an adjoint contribution `val` aimed at population i of the ghost cell
 * of `side` next to interior cell (k, j) (storage indices) to the interior
 * cell(s) that ghost value was made from at time t. */
static void ghost_adjoint(const kt_config* c, double* abar, int side, int i, int k, int j,
                          double along, double t, double val) {
    const kt_side* s = &c->side[side];
    int lo = along < s->split0 + s->split_speed * t;
    int kind = lo ? s->kind_lo : s->kind_hi;
    switch (kind) {
    case KT_PERIODIC:
        if (side == KT_LEFT) abar[at(c, i, k, c->nx)] += val;
        else if (side == KT_RIGHT) abar[at(c, i, k, 1)] += val;
        else if (side == KT_BOTTOM) abar[at(c, i, c->ny, j)] += val;
        else abar[at(c, i, 1, j)] += val;
        break;
    case KT_OUTFLOW:
        abar[at(c, i, k, j)] += val;
        break;
    case KT_REFLECT:
        abar[at(c, mirror(i, side == KT_LEFT || side == KT_RIGHT), k, j)] += val;
        break;
    default: /* Dirichlet: the ghost value does not depend on f */
        break;
    }
}

/* One adjoint step.  f: level-n state (its ghost layer is refilled for time
 * n dt); abar_next: adjoint of level n + 1 (interior of the ghost-layer
 * layout); abar: receives the adjoint of level n (same layout, ghosts zero).
 * *dtau accumulates sum_x sum_i abar_next_i(x) d out_i(x) / d tau with
 * d out_i / d tau = -(dt / tau^2) (f^eq_i - f_i). */
void kt_adjoint_step(const kt_config* c, double* f, long n, const double* abar_next,
                     double* abar, double* dtau) {
    double t = (double)n * c->dt;
    kt_fill_ghosts(c, f, t);
    size_t len = kt_field_len(c);
    for (size_t q = 0; q < len; ++q) abar[q] = 0.0;
    double coef[9][5];
    for (int i = 0; i < 9; ++i) star_coeffs(c, i, coef[i]);
    double w = c->dt / c->tau, acc_tau = 0.0;
    for (int k = 1; k <= c->ny; ++k)
        for (int j = 1; j <= c->nx; ++j) {
            double a[9], fc[9], J[81], m[4], feq[9];
            for (int i = 0; i < 9; ++i) {
                a[i] = abar_next[at(c, i, k, j)];
                fc[i] = f[at(c, i, k, j)];
            }
            /* collision: (dt / tau) J^T a */
            kt_feq_jacobian(c, fc, J);
            for (int jj = 0; jj < 9; ++jj) {
                double s = 0.0;
                for (int i = 0; i < 9; ++i) s += a[i] * J[i * 9 + jj];
                abar[at(c, jj, k, j)] += w * s;
            }
            /* tau */
            kt_moments(c, fc, m);
            kt_feq(c, m[0], m[1], m[2], m[3], feq);
            for (int i = 0; i < 9; ++i) acc_tau += a[i] * (-(c->dt / (c->tau * c->tau)) * (feq[i] - fc[i]));
            /* stencil links */
            double x = ((double)(j - 1) + 0.5) * c->dx, y = ((double)(k - 1) + 0.5) * c->dx;
            for (int i = 0; i < 9; ++i) {
                abar[at(c, i, k, j)] += coef[i][0] * a[i];
                if (j < c->nx) abar[at(c, i, k, j + 1)] += coef[i][1] * a[i];
                else ghost_adjoint(c, abar, KT_RIGHT, i, k, j, y, t, coef[i][1] * a[i]);
                if (j > 1) abar[at(c, i, k, j - 1)] += coef[i][2] * a[i];
                else ghost_adjoint(c, abar, KT_LEFT, i, k, j, y, t, coef[i][2] * a[i]);
                if (k < c->ny) abar[at(c, i, k + 1, j)] += coef[i][3] * a[i];
                else ghost_adjoint(c, abar, KT_TOP, i, k, j, x, t, coef[i][3] * a[i]);
                if (k > 1) abar[at(c, i, k - 1, j)] += coef[i][4] * a[i];
                else ghost_adjoint(c, abar, KT_BOTTOM, i, k, j, x, t, coef[i][4] * a[i]);
            }
        }
    *dtau += acc_tau;
}
