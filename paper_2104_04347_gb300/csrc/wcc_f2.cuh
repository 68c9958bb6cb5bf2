// wcc_f2.cuh -- a pair of FP32 lanes computed with Blackwell's paired FP32
// instructions (FADD2 / FMUL2 / FFMA2 through __fadd2_rn, __fmul2_rn,
// __ffma2_rn): one instruction does the same operation for two cells.  The
// generic scheme code (Cauchy-Kovalewski table, derivatives, eigenvectors)
// is instantiated with this type so that one thread advances two cells for
// the instruction cost of one.  Operations without a paired form (division,
// reciprocal, square root, min / max, comparisons) run lane by lane.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace wcc {

// keep the scalar math overloads visible next to the paired ones below
using ::fabs;
using ::fma;
using ::fmax;
using ::fmin;
using ::sqrt;

struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float2 x) : v(x) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    // broadcast of a scalar (constants of the scheme); explicit, so that
    // scalar expressions never turn into pairs by accident
    __device__ __forceinline__ explicit f2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ explicit f2(double a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ explicit f2(int a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
// (negations fold into the paired add as operand modifiers)
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { a = a + b; return a; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { a = a - b; return a; }
__device__ __forceinline__ f2& operator*=(f2& a, f2 b) { a = a * b; return a; }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
// Estimate of 1/a in each lane from the special-function unit (relative error
// about 2^-23): enough for quantities that only need FP32 accuracy.  For
// normal a only (densities); a subnormal a gives inf.
__device__ __forceinline__ f2 rcp_approx(f2 a) { return f2(__fdividef(1.f, a.v.x), __fdividef(1.f, a.v.y)); }
// 1/a to within an ulp: the estimate refined by one Newton-Raphson step,
// r + r (1 - a r), in paired instructions.
__device__ __forceinline__ f2 recip(f2 a) {
    const f2 r = rcp_approx(a);
    return fma(r, fma(-a, r, f2(1.f)), r);
}
__device__ __forceinline__ f2 fabs(f2 a) { return f2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ f2 fmin(f2 a, f2 b) { return f2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ f2 fmax(f2 a, f2 b) { return f2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
// a / b lane by lane.  Not a * (1/b): the limiter divides numbers that may
// both be subnormal (its epsilon defaults to 1e-40), whose reciprocal
// overflows although the quotient does not.
__device__ __forceinline__ f2 fdiv_fast(f2 a, f2 b) {
    return f2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}
__device__ __forceinline__ f2 rsqrt_approx(f2 a) { return f2(rsqrtf(a.v.x), rsqrtf(a.v.y)); }

// Helpers the generic scheme code uses for every real type.
template <class R>
constexpr bool is_f64 = std::is_same<R, double>::value;

__device__ __forceinline__ bool all_pos(double a) { return a > 0.0; }
__device__ __forceinline__ bool all_pos(float a) { return a > 0.f; }
__device__ __forceinline__ bool all_pos(f2 a) { return a.v.x > 0.f && a.v.y > 0.f; }
__device__ __forceinline__ float rsqrt_approx(float a) { return rsqrtf(a); }

}  // namespace wcc
