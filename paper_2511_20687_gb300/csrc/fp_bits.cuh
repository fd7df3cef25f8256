// FP64 <-> FP32 conversions by integer operations, shared by the FP64 kernels (hex8_math.cuh) and the
// double-float ones (df32.cuh).
#pragma once

#include <cuda_runtime.h>

namespace osam {
namespace hex8 {

// FP64 <-> FP32 with integer operations only.  GB300 executes the conversion instructions on its FP64
// pipe, the bound of every FP64 kernel here, so the hot paths rebuild the values from the IEEE-754
// layouts instead (sign kept, exponent re-biased between 1023 and 127, fraction cut to or widened
// from 23 bits).  f32_rz rounds toward zero (relative error below 2^-23); magnitudes below 2^-126
// become zero and beyond the FP32 range infinity (NaN too).  f64_of is exact for normal FP32 values
// and infinities; FP32 subnormals become zero.
__device__ __forceinline__ float f32_rz(double x) {
    const unsigned int hi = (unsigned int)__double2hiint(x);
    const unsigned int lo = (unsigned int)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned int frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned int mag = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : ((unsigned int)e << 23) | frac);
    return __uint_as_float((hi & 0x80000000u) | mag);
}
__device__ __forceinline__ double f64_of(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned int e = (b >> 23) & 0xffu;
    const unsigned int sign = b & 0x80000000u;
    if (e == 0) return __hiloint2double((int)sign, 0);
    const unsigned int ed = e == 255 ? 2047u : e + (1023u - 127u);
    return __hiloint2double((int)(sign | (ed << 20) | ((b & 0x7fffffu) >> 3)), (int)((b & 0x7u) << 29));
}

}  // namespace hex8
}  // namespace osam
