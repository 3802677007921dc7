// FP32 FMA throughput kernel: the denominator of the roofline of the
// ALU-bound Q1 element kernels, measured on the GPU that runs them.
//
// Every thread runs kChains independent FMA chains (enough independent work
// to cover the FMA latency at full occupancy), so the kernel is bound by the
// FP32 pipes alone; it reads nothing and writes one float per thread, so that
// the chains cannot be removed.  FLOPs = 2 * kChains * iters per thread.
#include <cuda_runtime.h>

#include "fem_b300.h"
#include "fem_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kCalibThreads = 256;

__global__ void __launch_bounds__(kCalibThreads) fma_rate_kernel(float* out, int iters) {
    const int tid = blockIdx.x * kCalibThreads + threadIdx.x;
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    const float x = 0.999999f, y = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[tid] = s;
}

}  // namespace

extern "C" {

fem_status fem_fp32_fma_rate(int blocks, int iters, float* out_dev, double* flops, void* stream) {
    if (blocks <= 0 || iters <= 0 || !out_dev) return femi::set_error(FEM_ERR_ARG, "fem_fp32_fma_rate: bad argument");
    fma_rate_kernel<<<blocks, kCalibThreads, 0, static_cast<cudaStream_t>(stream)>>>(out_dev, iters);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return femi::set_error(FEM_ERR_CUDA, cudaGetErrorString(e));
    if (flops) *flops = 2.0 * kChains * (double)iters * (double)blocks * kCalibThreads;
    return FEM_OK;
}

}  // extern "C"
