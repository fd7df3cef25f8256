// FP64 throughput probes (the denominators of the ALU rooflines of the FP64 kernels).
//   kind 0: fused multiply-adds on the FP64 pipe -- every thread runs 8 independent FMA chains held
//           in registers (2 flops per FMA);
//   kind 1: FP64 tensor-core MMA (mma.sync m8n8k4, 512 flops per warp instruction) -- every warp runs
//           4 independent accumulator chains;
//   kind 2: both in one kernel (the same warps interleave the chains of kinds 0 and 1), which shows
//           whether the two share one unit: if they do, its time is the sum of the other two.
// Each repeat is one launch of roughly 20 ms at the nominal rate, timed with CUDA events.
// The issue probe runs the FMA chains of kind 0 in one block (one SM) of `warps` warps with `lanes`
// active lanes each: the time per FP64 warp-instruction of one warp, the latency floor of element
// kernels on meshes too small to give every SM sub-partition several warps.
#include <cuda_runtime.h>

#include <vector>

#include "osam.h"
#include "osam_internal.h"

namespace osam {
namespace {

constexpr int kFmaChains = 8;
constexpr int kMmaChains = 4;

__device__ __forceinline__ void dmma_m8n8k4(double& d0, double& d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

template <bool FMA, bool MMA>
__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double seed, double* out) {
    double a[kFmaChains], c0[kMmaChains], c1[kMmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = seed + 1e-3 * (threadIdx.x + k);
#pragma unroll
    for (int k = 0; k < kMmaChains; ++k) { c0[k] = 1e-3 * k; c1[k] = -1e-3 * k; }
    const double m = 0.999999, c = 1e-7;
    const double fa = 1e-9 * (threadIdx.x & 7), fb = 1e-9 * (threadIdx.x >> 3);
    for (int it = 0; it < iters; ++it) {
        if (FMA) {
#pragma unroll
            for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], m, c);
        }
        if (MMA) {
#pragma unroll
            for (int k = 0; k < kMmaChains; ++k) dmma_m8n8k4(c0[k], c1[k], fa, fb);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
#pragma unroll
    for (int k = 0; k < kMmaChains; ++k) s += c0[k] + c1[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 FMA chains of kind 0 on the first `lanes` lanes of every warp of one block
__global__ void __launch_bounds__(1024) k_fp64_issue(int lanes, int iters, double* out) {
    double a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    const double m = 0.999999, c = 1e-7;
    if ((int)(threadIdx.x & 31) < lanes)
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], m, c);
        }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    out[threadIdx.x] = s;
}

// flops of one loop iteration of one 256-thread block
double block_iter_flops(int kind) {
    const double fma = 2.0 * kFmaChains * 256;
    const double mma = 512.0 * kMmaChains * (256 / 32);
    return kind == 0 ? fma : kind == 1 ? mma : fma + mma;
}

cudaError_t launch_probe(int kind, int blocks, int iters, double* out) {
    if (kind == 0) k_fp64_probe<true, false><<<blocks, 256>>>(iters, 1.0, out);
    else if (kind == 1) k_fp64_probe<false, true><<<blocks, 256>>>(iters, 1.0, out);
    else k_fp64_probe<true, true><<<blocks, 256>>>(iters, 1.0, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace osam

extern "C" OSAM_API int osam_fp64_probe(int device, int kind, int repeats, double* tflops, double* ms) {
    if (!tflops || repeats < 1 || repeats > 1000 || kind < 0 || kind > 2) return OSAM_EINVAL;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return OSAM_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return OSAM_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return OSAM_ECUDA;
    const int blocks = prop.multiProcessorCount * 8;
    // about 25 G flops per launch (20 ms at 1.25 TFLOP/s)
    const int iters = (int)(2.5e10 / (osam::block_iter_flops(kind) * blocks));
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * 256) != cudaSuccess) return OSAM_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t err = osam::launch_probe(kind, blocks, 64, out);  // warm-up
    for (int r = 0; r < repeats && err == cudaSuccess; ++r) {
        cudaEventRecord(e0);
        err = osam::launch_probe(kind, blocks, iters, out);
        cudaEventRecord(e1);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (err == cudaSuccess && t <= 0.f) err = cudaErrorUnknown;
        tflops[r] = osam::block_iter_flops(kind) * iters * (double)blocks / (t * 1e-3) / 1e12;
        if (ms) ms[r] = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return err == cudaSuccess ? OSAM_OK : OSAM_ECUDA;
}

// single-number FP64 FMA peak in GFLOP/s: the best of five probe launches
extern "C" OSAM_API int osam_fp64_peak(int device, double* gflops) {
    if (!gflops) return OSAM_EINVAL;
    double t[5];
    if (int rc = osam_fp64_probe(device, 0, 5, t, nullptr)) return rc;
    double best = 0.0;
    for (double x : t) best = x > best ? x : best;
    *gflops = best * 1e3;
    return OSAM_OK;
}

// time per FP64 warp-instruction of one warp when one block of `warps` warps (1..32) with `lanes`
// active lanes each (1..32) runs the FMA chains alone on one SM: best of three launches of ~20000
// iterations of 8 independent FMAs
extern "C" OSAM_API int osam_fp64_issue_probe(int device, int warps, int lanes, double* ns_per_instruction) {
    if (!ns_per_instruction || warps < 1 || warps > 32 || lanes < 1 || lanes > 32) return OSAM_EINVAL;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return OSAM_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return OSAM_ECUDA;
    const int threads = 32 * warps, iters = 20000;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * threads) != cudaSuccess) return OSAM_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    osam::k_fp64_issue<<<1, threads>>>(lanes, 64, out);   // warm-up
    cudaError_t err = cudaGetLastError();
    double best = 0.0;
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
        cudaEventRecord(e0);
        osam::k_fp64_issue<<<1, threads>>>(lanes, iters, out);
        cudaEventRecord(e1);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (err == cudaSuccess && t <= 0.f) err = cudaErrorUnknown;
        const double ns = t * 1e6 / ((double)iters * osam::kFmaChains);
        if (r == 0 || ns < best) best = ns;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *ns_per_instruction = best;
    return err == cudaSuccess ? OSAM_OK : OSAM_ECUDA;
}
