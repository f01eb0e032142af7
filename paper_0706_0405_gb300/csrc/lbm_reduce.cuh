// lbm_reduce.cuh -- block-wide FP64 reduction shared by the conservation
// kernels of liblbm (internal).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// Sum four doubles over the CTA (THREADS threads) in a fixed tree order, so
// the result does not depend on scheduling; every thread gets the totals in
// v.  sh: THREADS x 4 doubles of shared memory.
template <int THREADS>
__device__ __forceinline__ void block_sum4(double (&v)[4], double (*sh)[THREADS]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int s = THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = sh[q][0];
}

}  // namespace lbm
