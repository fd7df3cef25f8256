// Double-float ("f32x2") arithmetic on the FP32 pipes: a value is an unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from the error-free
// transformations of Knuth (TwoSum) and Dekker (FastTwoSum, TwoProduct via a fused multiply-add),
// as in the double-double literature (Dekker 1971; Hida, Li and Bailey 2001).  Every operation uses
// the _rn intrinsics so the compiler can neither contract a product into a later add nor reassociate:
// the transformations are only error-free when each operation is rounded exactly once.
#pragma once

#include <cuda_runtime.h>

#include "fp_bits.cuh"

namespace osam {
namespace df {

struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 make(float h, float l) { return f2{h, l}; }
__device__ __forceinline__ f2 one() { return f2{1.0f, 0.0f}; }

// s + e == a + b exactly
__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return f2{s, e};
}

// s + e == a + b exactly when |a| >= |b|
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return f2{s, e};
}

__device__ __forceinline__ f2 add(f2 a, f2 b) {
    f2 s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ f2 neg(f2 a) { return f2{-a.h, -a.l}; }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return add(a, neg(b)); }

__device__ __forceinline__ f2 mul(f2 a, f2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

// product of a double-float and a float
__device__ __forceinline__ f2 mulf(f2 a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return fast_two_sum(p, e);
}

// exact product of two floats
__device__ __forceinline__ f2 prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return f2{p, __fmaf_rn(a, b, -p)};
}

// a * b + c with one renormalisation: the product's error terms are folded into the sum's
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    f2 s = two_sum(p, c.h);
    s.l = __fadd_rn(s.l, __fadd_rn(e, c.l));
    return fast_two_sum(s.h, s.l);
}

// FP64 -> double-float and back with the integer conversions of fp_bits.cuh (the conversion
// instructions run on GB300's FP64 pipe): h = x cut to 24 bits, l = the exact remainder x - h cut to
// 24 bits (|x - (h + l)| < 2^-46 |x|), renormalised by FastTwoSum so that |l| <= ulp(h)/2 as the
// arithmetic above assumes; the way back is exact up to the final FP64 addition
__device__ __forceinline__ f2 from_double(double x) {
    const float h = hex8::f32_rz(x);
    return fast_two_sum(h, hex8::f32_rz(x - hex8::f64_of(h)));
}

__device__ __forceinline__ double to_double(f2 a) { return hex8::f64_of(a.h) + hex8::f64_of(a.l); }

// x^(-1/3) for x > 0: float seed, one Newton step y <- y + y (1 - x y^3) / 3 in double-float
// (the seed's relative error e becomes about 2 e^2, below the double-float rounding)
__device__ __forceinline__ f2 rcbrt(f2 x) {
    const float y0 = rcbrtf(x.h);
    const f2 y2 = prod(y0, y0);
    const f2 y3 = mulf(y2, y0);
    const f2 r = sub(one(), mul(x, y3));
    const f2 corr = mulf(r, __fmul_rn(y0, 1.0f / 3.0f));
    return add(f2{y0, 0.0f}, corr);
}

}  // namespace df
}  // namespace osam
