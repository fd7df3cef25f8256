// FP64 fused multiply-add throughput probe (the denominator of the ALU roofline of the FP64 element
// kernels): every thread runs 8 independent FMA chains held in registers.
#include <cuda_runtime.h>

#include "osam.h"
#include "osam_internal.h"

namespace osam {
namespace {

__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double seed, double* out) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + 1e-3 * (threadIdx.x + k);
    const double m = 0.999999, c = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace osam

extern "C" OSAM_API int osam_fp64_peak(int device, double* gflops) {
    if (!gflops) return OSAM_EINVAL;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return OSAM_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return OSAM_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return OSAM_ECUDA;
    const int blocks = prop.multiProcessorCount * 8, threads = 256, iters = 4096;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return OSAM_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    osam::k_fp64_fma<<<blocks, threads>>>(64, 1.0, out);  // warm-up
    cudaEventRecord(e0);
    osam::k_fp64_fma<<<blocks, threads>>>(iters, 1.0, out);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return OSAM_ECUDA;
    *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e6);
    return OSAM_OK;
}
