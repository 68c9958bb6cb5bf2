// wcc_convert.cuh -- per-value conversions between the host layout (FP64
// paper-scaled derivatives u_kx) and the FP32-mixed device planes (cell
// average as a float-float pair, Taylor coefficients e_k = u_kx / k! in FP32),
// written with FP32 and integer instructions only.
//
// GB300 executes FP64 arithmetic and FP64 <-> FP32 conversions at about 1/64
// of the FP32 rate, and a plain double-based conversion keeps its FP64 pipe
// busy for longer than the memory traffic takes.  Here instead:
//   * a double is split into floats hi + lo by integer operations on its bits
//     (hi = the leading 24 significant bits, lo = the remaining 29 bits
//     rounded to FP32);
//   * a float times a small integer (k!) is turned into a double exactly by
//     multiplying the 24-bit significand as an integer;
//   * the constant factors 1/k!, 1/((k+1)! 2^k) and 1/((k+1) 2^k) are applied
//     as float-float products, so the cell average keeps float-float accuracy
//     (a few units of 2^-48).
// Values outside the range where these are exact (zero aside: subnormal,
// tiny, huge, inf, NaN) take the hardware conversion, which is rare.  The
// doubles travel as 64-bit integers (their bit patterns): held as `double`,
// they kept the FP64 pipe two-thirds busy in the conversion kernels although
// no FP64 arithmetic ran.
#pragma once

#include <cuda_runtime.h>

#include "wcc_ff.cuh"

namespace wcc {

// A float-float constant: hi + lo rounds x to about 48 bits.
struct ffc {
    float hi, lo;
};
__host__ __device__ constexpr ffc ffc_of(double x) { return ffc{(float)x, (float)(x - (double)(float)x)}; }

// 1/k!, k = 0..6
__host__ __device__ constexpr ffc inv_fact_c(int k) {
    return k == 2 ? ffc_of(0.5) : k == 3 ? ffc_of(1.0 / 6.0) : k == 4 ? ffc_of(1.0 / 24.0)
         : k == 5 ? ffc_of(1.0 / 120.0) : k == 6 ? ffc_of(1.0 / 720.0) : ffc_of(1.0);
}
// weight of u_kx in the cell average, 1/((k+1)! 2^k) (Eq. SubEq:1DCellAVG; even k = 2, 4, 6)
__host__ __device__ constexpr ffc avg_from_u_c(int k) {
    return k == 2 ? ffc_of(1.0 / 24.0) : k == 4 ? ffc_of(1.0 / 1920.0) : ffc_of(1.0 / 322560.0);
}
// weight of e_k in the cell average, 1/((k+1) 2^k) (even k = 2, 4, 6)
__host__ __device__ constexpr ffc avg_from_e_c(int k) {
    return k == 2 ? ffc_of(1.0 / 12.0) : k == 4 ? ffc_of(1.0 / 80.0) : ffc_of(1.0 / 448.0);
}

__device__ __forceinline__ ff ff_mul_c(ff a, ffc c) { return ff_mul(a, ff{c.hi, c.lo}); }

// The rare cases, kept out of line: inlined, the compiler would predicate
// them into every call, and their FP64 instructions would occupy the FP64
// pipe even when predicated off.
static __device__ __noinline__ ff split_double_hw(double d) {
    ff r;
    split_double(d, r.hi, r.lo);
    return r;
}
static __device__ __noinline__ double float_times_hw(float f, double m) { return (double)f * m; }

// n < 2^29 rounded to the nearest float, without an integer-to-float
// conversion instruction (those run on the FP64 pipe of this GPU): each
// 23-bit part is read exactly as (2^23 + part) - 2^23, and one FMA joins them
// with a single rounding.
__device__ __forceinline__ float uint29_to_float(unsigned n) {
    const float lo = __uint_as_float(0x4B000000u | (n & 0x7fffffu)) - 8388608.f;
    const float hi = __uint_as_float(0x4B000000u | (n >> 23)) - 8388608.f;
    return fmaf(hi, 8388608.f, lo);
}

// The double with bit pattern b as hi + lo: hi = b truncated to 24
// significant bits, lo = the remaining bits rounded to FP32 (|lo| < ulp(hi));
// integer operations only for 2^-74 <= |d| < 2^128 and for zero.
__device__ __forceinline__ ff split_double_bits(unsigned long long b) {
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    if ((b << 1) == 0ull) return ff{__uint_as_float(sign), 0.f};
    const int e = (int)((b >> 52) & 0x7ffull) - 1023;
    if (e < -74 || e > 127) return split_double_hw(__longlong_as_double((long long)b));
    const unsigned long long mant = b & ((1ull << 52) - 1ull);
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
    // lo = +-rest * 2^(e - 52): rest (< 2^29) rounded to FP32, times a power of two
    const unsigned rest = (unsigned)(mant & ((1ull << 29) - 1ull));
    const float scale = __uint_as_float(sign | ((unsigned)(e - 52 + 127) << 23));
    return ff{hi, uint29_to_float(rest) * scale};
}

// floor(log2 m) for m >= 1
__host__ __device__ constexpr int ilog2c(unsigned m) { return m <= 1 ? 0 : 1 + ilog2c(m >> 1); }

// The bit pattern of f * M exactly as a double, for an integer 1 <= M <= 720:
// the 24-bit significand times M (< 2^34) renormalised with integer
// operations (its leading bit is 23 + floor(log2 M) or one above).
template <unsigned M>
__device__ __forceinline__ unsigned long long float_times_exact(float f) {
    static_assert(M >= 1 && M <= 720, "the product must fit the double's significand");
    constexpr int L0 = 23 + ilog2c(M);
    const unsigned u = __float_as_uint(f);
    if ((u << 1) == 0u) return (unsigned long long)u << 32;  // +-0
    const unsigned ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu)  // subnormal, inf, NaN
        return (unsigned long long)__double_as_longlong(float_times_hw(f, (double)M));
    const unsigned long long n = (unsigned long long)((u & 0x7fffffu) | 0x800000u) * M;
    const int lead = L0 + (int)(n >> (L0 + 1));  // n < 2^(L0 + 2)
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(lead + (int)ex - 150 + 1023) << 52) |
                                    ((n << (52 - lead)) & ((1ull << 52) - 1ull));
    return bits;
}

// The host-layout DOFs q[0..K-1] of one (cell, variable) -> the device
// values: the cell average ubar = sum over even k of q_k / ((k+1)! 2^k) as a
// float-float (normalised), and e_k = q_k / k! rounded to FP32, k >= 1.
template <int K>
__device__ __forceinline__ ff host_to_mixed(const unsigned long long* q, float (&e)[K]) {
    ff u = split_double_bits(q[0]);
#pragma unroll
    for (int k = 1; k < K; ++k) {
        const ff qk = split_double_bits(q[k]);
        e[k] = ff_mul_c(qk, inv_fact_c(k)).hi;
        if ((k & 1) == 0) u = ff_add(u, ff_mul_c(qk, avg_from_u_c(k)));
    }
    return fast_two_sum(u.hi, u.lo);
}

// The device values of one (cell, variable) -> host-layout DOFs (bit
// patterns): q_k = e_k k! (exact), q_0 = ubar - sum over even k of
// e_k / ((k+1) 2^k) (float-float, then one FP64 add to form the double).
template <int K>
__device__ __forceinline__ void mixed_to_host(ff ubar, const float (&e)[K], unsigned long long* q) {
    ff u = ubar;
#pragma unroll
    for (int k = 1; k < K; ++k) {
        q[k] = k == 2 ? float_times_exact<2>(e[k]) : k == 3 ? float_times_exact<6>(e[k])
               : k == 4 ? float_times_exact<24>(e[k]) : k == 5 ? float_times_exact<120>(e[k])
               : k == 6 ? float_times_exact<720>(e[k]) : float_times_exact<1>(e[k]);
        if ((k & 1) == 0) u = ff_sub(u, ff_mul_c(ff{e[k], 0.f}, avg_from_e_c(k)));
    }
    q[0] = (unsigned long long)__double_as_longlong(
        __longlong_as_double((long long)float_times_exact<1>(u.hi)) +
        __longlong_as_double((long long)float_times_exact<1>(u.lo)));
}

}  // namespace wcc
