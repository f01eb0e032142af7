/*
 * lbm.h -- C ABI of liblbm, a GB300 (sm_103a) implementation of the
 * Kataoka-Tsutahara two-dimensional nine-velocity (D2V9) finite-difference
 * lattice Boltzmann model with the added dissipation term of
 * Pan, Xu, Zhang & Jiang, "Lattice Boltzmann Approach to High-Speed
 * Compressible Flows", Int. J. Mod. Phys. C (2007).
 *
 * One call of lbm_step advances every interior node by one time step of
 * Eq. (SEC-VON-11):
 *   f_i(x, t + dt) = f_i - dt v_ia d_a f_i + dt lambda_i sum_a d_a^2 f_i
 *                    + (dt / tau) (f_i^eq - f_i),
 * with the moments of Eqs. (e4), (e5), (e7), the equilibrium of
 * Eqs. (e16)-(e18), the beta-upwind first derivative of Eqs. (SEC-VON-2a/2b)
 * and central second derivatives (Sec. 3, after Eq. SEC-VON-11).
 *
 * Conventions (all entry points)
 *  - Non-dimensional units with R = 1, so P = rho T; b = 2 / (gamma - 1).
 *  - Velocities (Eq. e14): v_0 = 0; v_1..4 = c1 (-1,0), (0,-1), (1,0), (0,1);
 *    v_5..8 = (c2 / sqrt 2) (-1,-1), (1,-1), (1,1), (-1,1); eta_0 = eta0,
 *    eta_1..8 = 0 (Eq. e15).  The diagonal pairs are read as c2 (cos, sin).
 *  - Cell-centred grid, dx = dy: node (ix, iy) sits at ((ix + 1/2) dx,
 *    (iy + 1/2) dx), 0 <= ix < nx, 0 <= iy < ny.
 *  - Field arrays (rho, ux, uy, T) are row-major ny x nx (index iy * nx + ix).
 *    Distribution arrays are 9 x ny x nx (index (i * ny + iy) * nx + ix).
 *    Their element type is the storage type of the context: double for
 *    LBM_FP64, float for the FP32 modes.
 *  - Pointers passed in may be device memory (cudaMalloc, torch CUDA
 *    tensors) or host memory (pageable or pinned); the library tells them
 *    apart with cudaPointerGetAttributes and stages host data through a
 *    buffer it owns.  Device inputs are read in place.  The caller owns every
 *    pointer it passes; the library never frees caller memory.
 *  - Work is queued on the context's stream.  Calls that return data to the
 *    host (lbm_sync, lbm_conservation, host outputs of lbm_moments,
 *    lbm_get_f, lbm_save) synchronise that stream before returning.
 *  - Errors: every call returns an lbm_status; nothing is thrown across the
 *    ABI.  lbm_last_error gives a message for the last failing call.
 *  - Health flags (sticky, cleared by lbm_init / lbm_set_f / lbm_load) record
 *    what the kernels saw in the levels they read: LBM_FLAG_NONPHYSICAL
 *    (rho <= 0 or a non-finite moment at some node) makes the next
 *    synchronising call return LBM_E_NONPHYSICAL; LBM_FLAG_T_NONPOSITIVE
 *    (T <= 0 at some node) is informational only: the scheme passes through
 *    short episodes of T < 0 right behind strong shocks (e.g. the 1000:1 tube
 *    of Eq. Riemann-2 with the Fig. 10 constants) and recovers.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_E_INVAL = -1,        /* an argument is out of range (message says which) */
    LBM_E_NOMEM = -2,        /* device or host allocation failed */
    LBM_E_CUDA = -3,         /* a CUDA runtime call or kernel launch failed */
    LBM_E_NONPHYSICAL = -4,  /* a level had rho <= 0 or a non-finite moment */
    LBM_E_TIMEOUT = -5,      /* a bounded device wait gave up */
    LBM_E_STATE = -6         /* call out of order (e.g. lbm_step before lbm_init) */
} lbm_status;

/* Bits of lbm_health. */
enum {
    LBM_FLAG_NONPHYSICAL = 1,   /* rho <= 0 or NaN / Inf in a moment */
    LBM_FLAG_TIMEOUT = 2,       /* a bounded device wait gave up */
    LBM_FLAG_T_NONPOSITIVE = 4  /* T <= 0 at some node (allowed, informational) */
};

/* Storage and arithmetic precision of a context.
 * LBM_FP32, LBM_FP32_T64 and LBM_FP32_TDF recover T from the internal energy
 * formed around u, T = sum_i f_i (|v_i - u|^2 + eta_i^2) / (b rho), so no
 * large totals cancel.
 * The modes marked "moment-exact" also correct the relaxation term
 * omega f^eq so that it carries exactly omega times the mass, momentum and
 * energy of f: an FP32 evaluation of f^eq loses them at high Mach (the
 * internal energy is a small part of terms of size u^2) and, the same loss
 * recurring every step, T drifts (tens of per cent over 5.8e4 steps of the
 * Mach-30 tube of Eq. Riemann-1 in LBM_FP32). */
typedef enum lbm_precision {
    LBM_FP64 = 0,      /* f stored and updated in FP64 */
    LBM_FP32 = 1,      /* f in FP32; internal energy summed in FP32 */
    LBM_FP32_T64 = 2,  /* f in FP32; internal energy accumulated in FP64;
                          moment-exact */
    LBM_FP32_TDF = 3,  /* f in FP32; internal energy in double-float (pairs
                          of FP32 with error-free sums and products);
                          moment-exact */
    LBM_FP32_CONS = 4  /* f in FP32; T = (E / rho - u^2) / b in FP32 (at
                          high Mach its cancellation costs ~2^-24 u^2 / T
                          relative in T, which only shapes the equilibrium:
                          the mass, momentum and energy are kept by the
                          moment-exact relaxation); moment-exact */
} lbm_precision;

/* Boundary kinds.  The paper names the kinds (Sec. 4.2, text of
 * Eq. Riemann-3) but not how they act on f; the library uses one ghost layer:
 *   PERIODIC  ghost = the node at the opposite edge (both opposite sides
 *             must be PERIODIC and unsplit);
 *   OUTFLOW   zero gradient: ghost = the adjacent interior node;
 *   DIRICHLET ghost = f^eq of the side's state (rho, ux, uy, T);
 *   REFLECT   specular wall halfway between ghost and edge node: ghost_i =
 *             f_m(i) of the adjacent node, m reversing the wall-normal
 *             velocity component. */
typedef enum lbm_bc_kind {
    LBM_BC_PERIODIC = 0,
    LBM_BC_OUTFLOW = 1,
    LBM_BC_DIRICHLET = 2,
    LBM_BC_REFLECT = 3
} lbm_bc_kind;

enum { LBM_SIDE_LEFT = 0, LBM_SIDE_RIGHT = 1, LBM_SIDE_BOTTOM = 2, LBM_SIDE_TOP = 3 };

/* One side of the rectangle.  The side may switch kind at the along-side
 * coordinate s(t) = split0 + split_speed * t (x for bottom/top, y for
 * left/right, cell-centre coordinates): ghost cells whose centre lies below
 * s(t) use kind_lo / state_lo, the others kind_hi / state_hi.  Use
 * split0 = +INFINITY for an unsplit side.  t is the time of the level whose
 * ghosts are filled (step index times dt).  This expresses the
 * double-Mach-reflection wall start and its moving exact shock position on
 * the top boundary (Sec. 4.2, Fig. 12). */
typedef struct lbm_bc {
    int kind_lo;
    int kind_hi;
    double split0;
    double split_speed;
    double state_lo[4]; /* (rho, ux, uy, T) for DIRICHLET below the split */
    double state_hi[4]; /* ... above the split */
} lbm_bc;

/* DVM constants of Eqs. (e14), (e15): c1, c2 > 0, c1 != c2 (Eqs. e17, e18
 * divide by c1^2 - c2^2), eta0 > 0. */
typedef struct lbm_dvm {
    double c1, c2, eta0;
} lbm_dvm;

/* Scheme parameters: beta in [0, 1/2] (Eqs. SEC-VON-2a/2b; 0 = first-order
 * upwind, 1/2 = central) and the dissipation coefficients lambda_i >= 0 of
 * Eq. (SEC-VON-11) (Eq. SEC-VON-13 suggests c1 dx, c1 dx / 10 (i = 1..4),
 * 0 (i = 5..8)). */
typedef struct lbm_dissipation {
    double beta;
    double lambda[9];
} lbm_dissipation;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of one level buffer of a context for an nx x ny grid in precision
 * prec: (ny + 2) x 9 x pitch elements of the storage type, pitch = nx + 8
 * rounded up to a multiple of 32.  0 for nx, ny outside [1, 2^24] or an
 * unknown precision.  Needs no GPU. */
size_t lbm_level_bytes(int nx, int ny, lbm_precision prec);

/* Create a context for an nx x ny grid (nx, ny >= 1).  b > 0, tau > 0,
 * dt > 0, dx > 0; the collision factor per step is dt / tau (Eq. SEC-VON-1
 * with dt equal to the Knudsen number, Sec. 2).  bc[4] in LBM_SIDE_* order.
 * stream: a cudaStream_t (NULL = the legacy default stream) on the current
 * device, which the context keeps using.
 * The state f of Eq. (SEC-VON-1) lives in two level buffers (the current
 * level and the next, alternating), each lbm_level_bytes(nx, ny, prec) bytes
 * in the library's internal layout: row-interleaved, grid row iy + 1 (rows 0
 * and ny + 1 are ghost rows) holding the nine population rows of that grid
 * row one after the other, node (ix, iy) at column ix + 4 of each.
 *  - f_buf0 = f_buf1 = NULL: the context allocates both and frees them in
 *    lbm_destroy.
 *  - Both non-NULL: the caller's device memory (e.g. two torch CUDA tensors
 *    from its own allocator), on the current device, each 256-byte aligned
 *    and at least lbm_level_bytes long, not overlapping.  The context zeroes
 *    them here, keeps stepping in them and never frees them; they must stay
 *    allocated until lbm_destroy returns, and the caller must not write them
 *    while the context's stream has work queued.  After lbm_destroy they
 *    still hold the last levels.  Exactly one NULL, a misaligned or
 *    overlapping pair, or memory that is not device memory of the current
 *    device gives LBM_E_INVAL.
 * On failure *out is NULL and lbm_last_error(NULL) explains. */
lbm_status lbm_create(int nx, int ny, double b, double tau, double dt, double dx,
                      const lbm_dvm* dvm, const lbm_dissipation* diss, const lbm_bc bc[4],
                      lbm_precision prec, void* stream, void* f_buf0, void* f_buf1, lbm_ctx** out);

/* Free everything the context owns (waits for its stream first). NULL is a
 * no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last failing call on ctx (ctx = NULL: the last failing
 * lbm_create of this thread).  Never NULL; valid until the next call. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Initial condition f_i = f_i^eq(rho, ux, uy, T) (Eqs. e16-e18) at every node,
 * ghost layer filled for t = 0; the step counter is reset to 0.  Fields are
 * ny x nx arrays of the storage type; rho > 0 and T > 0 are the caller's
 * responsibility (a violation shows as LBM_E_NONPHYSICAL later). */
lbm_status lbm_init(lbm_ctx* ctx, const void* rho, const void* ux, const void* uy,
                    const void* T);

/* Advance n >= 0 steps of Eq. (SEC-VON-11), asynchronously on the stream.
 * Each step reads level k, writes level k + 1 into the other buffer and fills
 * that level's ghost layer for t = (k + 1) dt in the same kernel. */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* Macroscopic fields of the current level (Eqs. e4, e5, e7): rho, ux, uy, T
 * as ny x nx arrays of the storage type.  Any output may be NULL (skipped). */
lbm_status lbm_moments(lbm_ctx* ctx, void* rho, void* ux, void* uy, void* T);

/* FP64 totals over the interior of the current level: out[0] = sum rho,
 * out[1] = sum rho ux, out[2] = sum rho uy, out[3] = sum rho (b T + u^2)
 * (the sums of Eqs. e4, e5, e7).  Deterministic (fixed reduction order).
 * out is host memory; synchronises. */
lbm_status lbm_conservation(lbm_ctx* ctx, double out[4]);

/* Wait for the stream; returns LBM_E_NONPHYSICAL / LBM_E_TIMEOUT if the
 * corresponding health flag is set. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Wait for the stream and store the sticky LBM_FLAG_* bits in *flags (host). */
lbm_status lbm_health(lbm_ctx* ctx, unsigned* flags);

/* Copy the current level's interior distribution (9 x ny x nx, storage type)
 * to dst / set it from src (then fill the ghost layer for t = step * dt and
 * set the step counter to `step`). */
lbm_status lbm_get_f(lbm_ctx* ctx, void* dst);
lbm_status lbm_set_f(lbm_ctx* ctx, const void* src, long long step);

/* Step index of the current level. */
long long lbm_step_count(const lbm_ctx* ctx);

/* Checkpoint: lbm_checkpoint_bytes gives the size; lbm_save writes a header
 * (grid, precision, step) and the interior distribution to buf (host or
 * device); lbm_load restores it (LBM_E_INVAL if the header does not match
 * the context). */
size_t lbm_checkpoint_bytes(const lbm_ctx* ctx);
lbm_status lbm_save(lbm_ctx* ctx, void* buf, size_t bytes);
lbm_status lbm_load(lbm_ctx* ctx, const void* buf, size_t bytes);

/* ------------------------------------------------------------- adjoint
 * The adjoint of lbm_step is the transpose of the linearised update of
 * Eq. (SEC-VON-11): the transposed five-point star, the ghost links routed
 * back through the boundary rule (outflow and reflect feed the edge node,
 * periodic wraps, Dirichlet feeds nothing) and the transposed Jacobian of
 * f -> f^eq(moments(f)) (Eqs. e4, e5, e7, e16-e18).  Adjoint arrays are
 * dense 9 x ny x nx of the storage type (FP32 contexts use an FP32 adjoint).
 *
 * lbm_record(ctx, K): keep a copy of the current level now and of every K-th
 * level lbm_step produces from here (K = 0 stops recording); memory grows by
 * one level per K steps.  lbm_init / lbm_set_f / lbm_load stop recording. */
lbm_status lbm_record(lbm_ctx* ctx, int every);

/* Seed the adjoint of the current level from adjoints of its moments:
 * abar_j = sum_m qbar_m d q_m / d f_j with q = (rho, ux, uy, T); any qbar may
 * be NULL (zero).  qbar are ny x nx fields, abar a 9 x ny x nx output. */
lbm_status lbm_adjoint_seed(lbm_ctx* ctx, const void* qbar_rho, const void* qbar_ux,
                            const void* qbar_uy, const void* qbar_T, void* abar);

/* Apply n adjoint steps: abar (in: adjoint of the current level k; out:
 * adjoint of level k - n).  Levels are recomputed from the checkpoint that
 * starts each segment of K steps (memory K + 2 levels besides the
 * checkpoints).  *dL_dtau (host, may be NULL) is incremented by the tau
 * derivative of these n steps, d out_i / d tau = -(dt / tau^2) (f^eq_i - f_i).
 * Afterwards the context's current level is k - n.  LBM_E_STATE without a
 * recording, LBM_E_INVAL if fewer than n steps are recorded. */
lbm_status lbm_adjoint_step(lbm_ctx* ctx, int n, void* abar, double* dL_dtau);

/* Gradient with respect to the fields of an initial condition f = f^eq(q):
 * g_m = sum_i abar_i d f^eq_i / d q_m at the fields q = (rho, ux, uy, T);
 * any output may be NULL. */
lbm_status lbm_feq_vjp(lbm_ctx* ctx, const void* rho, const void* ux, const void* uy, const void* T,
                       const void* abar, void* g_rho, void* g_ux, void* g_uy, void* g_T);

/* Launch shape of the step kernel. */
typedef struct lbm_launch {
    int variant; /* 0: one thread per node, neighbours read through L1/L2;
                    1: FP32 modes only: CTAs own column strips and march up a
                    balanced run of rows, rows of all nine planes staged in a
                    shared-memory ring by bulk asynchronous copies;
                    2: FP32 modes only: each thread updates tx x-adjacent
                    nodes with vector loads and stores;
                    3: FP32 modes only (default): persistent CTAs of 128
                    threads, two x-adjacent nodes each; each 64 x 4 tile plus
                    its halo (72 x 6 x 9 planes) arrives in shared memory by
                    one tiled tensor copy (TMA), double-buffered, and the
                    stencil reads shared memory */
    int tx;      /* variant 1: columns per CTA, 128 or 256; variant 2: 2 or 4 */
    int ring;    /* variant 1: ring slots, 4 or 6 (4 when tx = 128) */
    int grid;    /* variants 1, 3: CTAs; 0 = one full wave (SMs x resident CTAs) */
} lbm_launch;

/* Set / read the launch shape used by lbm_step (LBM_E_INVAL for shapes the
 * library does not have; variant 1 on an FP64 context is rejected). */
lbm_status lbm_set_launch(lbm_ctx* ctx, const lbm_launch* launch);
lbm_status lbm_get_launch(const lbm_ctx* ctx, lbm_launch* launch);

/* Time every available launch shape for `steps` steps each (CUDA events on
 * the context's stream, after one untimed step), keep the fastest, and
 * restore the state and step counter the context had before.  Writes the
 * chosen shape to *best (may be NULL) and the per-step milliseconds of each
 * candidate to ms[0..n) if ms is not NULL (n = the number of candidates,
 * at most 8, stored in *n_candidates if not NULL).  Candidates, in order:
 * variant 0; for FP32 also (3), (2, 4), (2, 2), (1, 256, 4), (1, 256, 6),
 * (1, 128, 4). */
lbm_status lbm_autotune(lbm_ctx* ctx, int steps, lbm_launch* best, double* ms, int* n_candidates);

/* FP64 conservation totals (out[0..3] = sum rho, sum rho ux, sum rho uy,
 * sum rho (b T + u^2), the quantities of lbm_conservation; the two sum in
 * different orders, so they agree to rounding, about 1e-15 relative, not
 * bit for bit) of a dense 9 x ny x nx
 * distribution f in device memory (the layout lbm_get_f writes; element type
 * double for LBM_FP64, float for the FP32 modes), for callers that cannot
 * allocate device memory: a process whose device memory is committed to a
 * fixed pool or a framework's caching allocator, a latency-critical loop in
 * which an allocation could synchronise and stall the device, a host with a
 * fixed device-memory budget.  No context is needed and nothing is
 * allocated.  The paper has no counterpart; this is a service of the library.
 *  - Scratch: a fixed device array inside the library (64 KiB + 32 B), held on
 *    every GPU that loads the library until the process exits.  It bounds
 *    nx * ny to 8 388 608 nodes (2048 tiles of 4096); larger grids get
 *    LBM_E_INVAL.
 *  - The first call in each CUDA context (normally once per device, in the
 *    runtime's primary context) looks up that array's device address in
 *    that context, with the device current, and keeps it under the
 *    context's unique ID; a non-primary context, or a new primary context
 *    after cudaDeviceReset, does its own look-up.
 *  - All calls share the array; calls that overlap on the GPU race and may
 *    return wrong totals.  Each call writes every value it reads, so a call
 *    never depends on an earlier call's contents.
 *  - Work runs on `stream` (a cudaStream_t, NULL = legacy default stream),
 *    after whatever the caller queued there; the call synchronises that
 *    stream and writes out (host or device memory) before returning.
 *  - Errors: LBM_E_INVAL (NULL pointer, nx or ny < 1, too many nodes, unknown
 *    precision), LBM_E_CUDA (launch or copy failed).  lbm_last_error does not
 *    describe errors of this call. */
lbm_status lbm_conservation_noalloc(const void* f, int nx, int ny, lbm_precision prec,
                                    const lbm_dvm* dvm, double out[4], void* stream);

/* --------------------------------------------------------------- batch
 * Many independent problems (each with its own grid, constants and boundary
 * kinds) advanced together by one persistent cooperative kernel launch per
 * lbm_batch_step call: every CTA walks a contiguous share of the list of
 * (problem, 64 x 4 node tile) pairs each step, and starts a step once the
 * CTAs owning the tiles next to its own have finished the previous one
 * (bounded waits, LBM_E_TIMEOUT if one gives up; see lbm_batch_plant_stall
 * below).  The launch is captured
 * once per step count into a CUDA graph on a stream private to the batch and
 * replayed there, ordered after the batch's stream by events (so the legacy
 * default stream works too); if capture fails the launch runs directly.  The per-node
 * arithmetic is that of lbm_step, so every problem's levels equal those of
 * stepping it alone.  FP32 modes only. */
typedef struct lbm_problem {
    int nx, ny;
    double b, tau, dt, dx;
    lbm_dvm dvm;
    lbm_dissipation diss;
    lbm_bc bc[4];
} lbm_problem;

typedef struct lbm_batch lbm_batch;

lbm_status lbm_batch_create(int nprob, const lbm_problem* probs, lbm_precision prec, void* stream,
                            lbm_batch** out);
void lbm_batch_destroy(lbm_batch* batch);
const char* lbm_batch_last_error(const lbm_batch* batch);

/* rho[p], ux[p], uy[p], T[p]: problem p's ny x nx fields (float); every
 * problem is initialised and the batch's step counter reset to 0. */
lbm_status lbm_batch_init(lbm_batch* batch, const void* const* rho, const void* const* ux,
                          const void* const* uy, const void* const* T);

/* Advance every problem n steps (asynchronous). */
lbm_status lbm_batch_step(lbm_batch* batch, int n);

/* Wait; LBM_E_NONPHYSICAL / LBM_E_TIMEOUT as for lbm_sync. */
lbm_status lbm_batch_sync(lbm_batch* batch);

/* The context of problem p (owned by the batch; use it for lbm_moments,
 * lbm_get_f, lbm_conservation ... after lbm_batch_sync; do not destroy it). */
lbm_ctx* lbm_batch_problem(lbm_batch* batch, int p);

/* Launch facts: CTAs of the persistent launch, tiles per step, and 1 if the
 * last lbm_batch_step ran from a CUDA graph (0 before any step, -1 if graph
 * capture failed and the launch runs directly). */
lbm_status lbm_batch_info(const lbm_batch* batch, int* grid, int* ntiles, int* graph);

/* Launch shape of the batch kernel: npt = nodes per thread (1: 256-thread
 * CTAs, one node each; 2: 128-thread CTAs, two x-adjacent nodes each, 8-byte
 * shared-memory accesses) and grid = CTAs of the cooperative launch (1 up to
 * the resident CTAs of a full wave, capped at the work-item count; 0 = a
 * full wave).  block = 3, 5 or 7 selects temporal blocking instead (only for
 * batches whose problems all have at most 8 rows and no periodic x sides):
 * one pass advances a 128-column segment of a problem by `block` steps in
 * shared memory (halo of `block` columns each side, recomputed), so DRAM
 * traffic and grid barriers drop by that factor; npt is then ignored.
 * block = 0 or 1 is the one-step tile kernel.  Every shape computes the same
 * bits.  Setting a shape drops the captured graph (the next lbm_batch_step
 * captures a new one). */
typedef struct lbm_batch_launch {
    int npt;
    int grid;
    int block;
} lbm_batch_launch;

lbm_status lbm_batch_set_launch(lbm_batch* batch, const lbm_batch_launch* launch);
lbm_status lbm_batch_get_launch(const lbm_batch* batch, lbm_batch_launch* launch);

/* Time each candidate shape -- npt 1 and 2, each with a full wave and half a
 * wave of CTAs, then (where the batch allows it) temporal blocking with 3, 5
 * and 7 steps per pass on a full wave -- for `steps` steps on the batch's own
 * current state (after one untimed step per shape), restore the state, the
 * level counter and the health flags, and keep the fastest.  best (may be
 * NULL) receives it; ms[0..n) (may be NULL, room for 8) the per-step
 * milliseconds of each candidate in that order; *n_candidates (may be NULL)
 * their number.
 * Allocates one copy of every problem's current level for the duration of
 * the call; synchronises the batch's stream. */
lbm_status lbm_batch_autotune(lbm_batch* batch, int steps, lbm_batch_launch* best, double* ms,
                              int* n_candidates);

/* Step ordering inside the one-step tile kernel: a CTA starts step s + 1 as
 * soon as every CTA owning a tile next to one of its own (periodic partners
 * included) has finished step s, rather than at a grid-wide barrier; one
 * grid barrier ends each launch.  (A grid barrier after every step remains
 * for launch shapes whose neighbour lists would be longer than 8 CTAs.)
 * Every such wait, like the grid barriers, gives up after a bound: the
 * launch then stops, and the next lbm_batch_sync returns LBM_E_TIMEOUT;
 * lbm_batch_init makes the batch usable again.
 *
 * lbm_batch_set_wait_limit: that bound in seconds, (0, 60], for every batch
 * of the current device (default 2 s); converted to SM cycles at the
 * device's nominal clock.  LBM_E_INVAL outside the range.
 *
 * lbm_batch_plant_stall: failure injection for tests, on the host side.
 * cta in [0, grid) adds to that CTA's neighbour list a counter that no CTA
 * ever advances, so its wait before its second step of the next launch runs
 * out (after the bound above) and the launch reports LBM_E_TIMEOUT; nothing
 * faults or hangs.  cta < 0 restores the lists.  LBM_E_STATE if the current
 * launch shape has no neighbour lists (temporal blocking, or lists too long);
 * LBM_E_INVAL for cta >= grid.  Synchronises the batch's stream. */
lbm_status lbm_batch_set_wait_limit(double seconds);
lbm_status lbm_batch_plant_stall(lbm_batch* batch, int cta);

/* Failure injection for tests, on the host side: after `after` more device
 * allocations by the library succeed, the next one fails as if the device
 * were out of memory (and the countdown stops); after < 0 switches it off.
 * The failing call returns LBM_E_NOMEM and frees what it had allocated.
 * Process-wide; always LBM_OK. */
lbm_status lbm_inject_alloc_failure(long long after);

/* -------------------------------------------------- von Neumann scanner
 * Linear stability of the scheme about a uniform state (Sec. 3): a Fourier
 * mode exp(i k.x) of a perturbation of f is multiplied each step by the 9 x 9
 * amplification matrix of Eqs. (SEC-VON-8, SEC-VON-12),
 *   G(k) = diag(W_i(k)) + (dt / tau) d f^eq / d f,
 * with W_i(k) the symbol of the step's five-point stencil for velocity i
 * (beta-upwind advection of Eqs. SEC-VON-2a/2b, the lambda_i Laplacian and
 * the -dt/tau of the relaxation) and d f^eq / d f the Jacobian of the
 * equilibrium of the moments at the state (Eqs. e4, e5, e7, e16-e18).  The
 * scheme damps every mode when the spectral radius max|eig G| <= 1 (Figs.
 * 2-7 plot it against k dx).
 *
 * One case: the constants a context would get from lbm_create and the
 * uniform state (rho, ux, uy, T). */
typedef struct lbm_vn_case {
    double b, tau, dt, dx;
    lbm_dvm dvm;
    lbm_dissipation diss;
    double state[4];
} lbm_vn_case;

/* For every case c, direction d and m = 0 .. nk - 1, the spectral radius of
 * G(k) at k dx = (pi m / (nk - 1)) (dirs[2d], dirs[2d + 1]) (k = 0 when
 * nk = 1; the paper scans k dx from 0 to pi in 31 points along x):
 *   radius[(c * ndirs + d) * nk + m]      (ncases x ndirs x nk doubles)
 *   growth[c] = max over d and m          (ncases doubles)
 * The eigenvalues come from a Hessenberg reduction and the shifted QR
 * iteration in FP64, one matrix per GPU thread; an entry is NaN if the
 * iteration did not converge in 60 sweeps per eigenvalue (growth is then NaN).
 *  - cases (ncases) and dirs (2 x ndirs ints, each pair in [-1024, 1024] and
 *    not (0, 0), e.g. (1,0), (0,1), (1,1), (1,-1)) are host memory, read
 *    before the call returns.
 *  - radius and growth may each be NULL (not both), device memory (written
 *    asynchronously on `stream`) or host memory (the call then synchronises
 *    `stream`).  The caller owns them.
 *  - stream: a cudaStream_t (NULL = the legacy default stream).  The call
 *    allocates its scratch (81 doubles per case, plus radius when that is not
 *    in device memory) with cudaMallocAsync on that stream and frees it in
 *    stream order.
 *  - ncases = 0 does nothing.  LBM_E_INVAL: ncases < 0, NULL cases / dirs,
 *    ndirs outside [1, 64], nk outside [1, 65536], ncases * ndirs * nk
 *    >= 2^31, or a case with b, tau, dt, dx, c1, c2, eta0 not finite and > 0,
 *    c1 == c2, beta outside [0, 1/2], a negative lambda, rho or T not > 0
 *    (the message, from lbm_last_error(NULL), names the case).  LBM_E_NOMEM /
 *    LBM_E_CUDA if the scratch or a launch fails. */
lbm_status lbm_vn_scan(const lbm_vn_case* cases, int ncases, const int* dirs, int ndirs, int nk,
                       double* radius, double* growth, void* stream);

/* FP64 and FP32 FMA throughput (TFLOP/s, 2 flops per FMA) of the current
 * device, from chains of dependent FMAs on every SM (~0.1 s).  Not from the
 * paper: the benchmark's ceiling for the FP64 step, which is bounded by the
 * FP64 pipe rather than by HBM on this part. */
lbm_status lbm_probe_rates(double* fp64_tflops, double* fp32_tflops);

/* Data-movement ceiling of the FP32 tile step (LBM_STEP_TILE) on an nx x ny
 * grid: a kernel with the step kernel's tile walk, its tensor copies of the
 * 72 x 9 x 6 halo boxes of one level and its 8-byte stores of the other
 * level, but no arithmetic (each node's nine values are copied through).
 * *gbs = 72 bytes (nine FP32 values read and nine written) per node over
 * the best of `reps` launches (after two warm-up launches), alternating the
 * two levels.  Allocates and frees two levels of its own; synchronises.
 * Not from the paper: the benchmark reports the step kernel against it.
 * LBM_E_INVAL for nx, ny < 1, reps < 1 or gbs NULL; LBM_E_NOMEM; LBM_E_CUDA
 * (also when the tensor-copy interface is unavailable); LBM_E_TIMEOUT if a
 * bounded wait of the kernel gave up. */
lbm_status lbm_probe_tile_copy(int nx, int ny, int reps, double* gbs);

/* Version string of the library. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
