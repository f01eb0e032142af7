// lbm_launch.h -- host-side launchers of the liblbm kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// Kernel variant and launch shape of the step (chosen by the host, see
// lbm_tune in lbm.h).
enum StepVariant : int { STEP_SIMPLE = 0, STEP_RING = 1 };
struct StepConfig {
    int variant = STEP_RING;  // FP64 always uses STEP_SIMPLE
    int tx = 256;             // ring: columns per CTA (128 or 256)
    int ring = 4;             // ring: shared-memory row slots (4 or 6; 4 when tx = 128)
    int grid = 0;             // ring: CTAs (0 = SMs x resident CTAs per SM)
};

// One step, level `level` in fin -> level + 1 in fout (ghosts included).
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

}  // namespace lbm
