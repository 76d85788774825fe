// Double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  Used where a
// long FP64 accumulation would otherwise run on the FP64 pipe, which on sm_103a issues
// at a small fraction of the FP32 rate.
//
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), the renormalising
// FastTwoSum for |a| >= |b| (Dekker 1971), and the FMA-based exact product
// a * b = p + fma(a, b, -p).  Products of two double-floats drop the lo * lo term
// (below 2^-48 relative).  Device code only.
#pragma once

#include <cuda_runtime.h>

namespace dotk {

struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_zero() { return dfloat{0.f, 0.f}; }

// Round an FP64 value to the nearest double-float (the low part carries the next 24
// bits of the significand).
__device__ __forceinline__ dfloat df_from(double x) {
    const float h = __double2float_rn(x);
    return dfloat{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat{-a.hi, -a.lo}; }

// s + e = a + b exactly (any magnitudes).
__device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = a + b;
    const float bv = s - a;
    const float av = s - bv;
    return dfloat{s, (a - av) + (b - bv)};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
    const float s = a + b;
    return dfloat{s, b - (s - a)};
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    dfloat s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);  // exact rounding error of the leading product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// acc + a * b
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat acc) { return df_add(acc, df_mul(a, b)); }

}  // namespace dotk
