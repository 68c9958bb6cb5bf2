// wcc_ff.cuh -- float-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA-based
// TwoProduct; the compound operations follow the usual "sloppy" double-word
// algorithms (e.g. Joldes, Muller & Popescu, ACM TOMS 2017), whose relative
// error is a small multiple of 2^-48.  They rely on IEEE round-to-nearest
// FP32 adds without reassociation; contraction into FMA is harmless.
#pragma once

#include <cuda_runtime.h>

namespace wcc {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float h, float l) { return ff{h, l}; }

// s + e == a + b exactly (Knuth).
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

// s + e == a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

// p + e == a * b exactly.
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_add(ff a, float b) {
    ff s = two_sum(a.hi, b);
    const float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

// Split a double into a float-float (host or device).
__host__ __device__ __forceinline__ void split_double(double d, float& hi, float& lo) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
}

}  // namespace wcc
