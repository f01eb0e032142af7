// lbm_probe.cu -- lbm_probe_rates: FP64 and FP32 FMA throughput of the
// current device, measured by chains of dependent FMAs (8 independent chains
// per thread, 8 CTAs of 256 threads per SM).  The benchmark uses the FP64
// figure as the ceiling of the FP64 step, which is arithmetic-bound on parts
// whose FP64 rate is a small fraction of their FP32 rate.
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace {
constexpr int kIters = 4096;

template <typename T>
__global__ void k_fma_chains(T* out, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x * 1e-3 + k);
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // out holds gridDim.x * blockDim.x values
}

template <typename T>
double rate(T* buf, int blocks, int threads, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<blocks, threads, 0, st>>>(buf, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    return 2.0 * 8.0 * kIters * (double)blocks * threads / (best * 1e-3) / 1e12;
}
}  // namespace

extern "C" lbm_status lbm_probe_rates(double* fp64_tflops, double* fp32_tflops) {
    if (!fp64_tflops || !fp32_tflops) return LBM_E_INVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    const int threads = 256, blocks = sms * 8;
    double* buf = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status r = LBM_OK;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * threads) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        r = LBM_E_CUDA;
    } else {
        *fp64_tflops = rate<double>(buf, blocks, threads, st, e0, e1);
        *fp32_tflops = rate<float>(reinterpret_cast<float*>(buf), blocks, threads, st, e0, e1);
        if (*fp64_tflops < 0 || *fp32_tflops < 0) r = LBM_E_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    cudaGetLastError();
    return r;
}
