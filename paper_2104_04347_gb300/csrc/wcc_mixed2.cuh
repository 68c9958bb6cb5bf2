// wcc_mixed2.cuh -- the FP32-mixed half-step (no FP64 instruction in the
// per-cell work), two cells per thread.
//
// Storage per variable: the cell average ubar as a float-float pair (two FP32
// planes, hi and lo) and the Taylor coefficients e_1..e_P as FP32 planes
// (e_k = dx^k u^(k) / k!; the scaled form keeps them in range).  Arithmetic:
//   * float-float (compensated FP32) where a result is a small difference of
//     O(1) quantities or must conserve: the leading flux term f(u_0), each
//     parent's share A = ubar / 2 + lam fbar + dodd / 2 of its average, the
//     new cell average A[left] + (ubar - A)[right] (Eq. SubEq:1DIntegral);
//   * FP32 for everything else: the Cauchy-Kovalewski table, the higher flux
//     and vertex terms, derivatives, the limiter.  The vertex values enter
//     only as ubar - u_{i-1/2}, u_{i+1/2} - ubar (Eqs. SubEq:1DU12,
//     1DHighOrderWeights) and e_1, each formed from Sterbenz-exact
//     differences of float-float averages plus FP32 deviations.
// Because the limited polynomial keeps the cell average (Eq.
// 1DLimitedPolynomial), the limiter works on deviations from ubar only and
// never rounds ubar; sums of ubar telescope up to float-float rounding.  The
// limiter weights are evaluated in a scale-free form (ratios to the smallest
// denominator), so the tiny epsilon of the paper neither overflows nor
// underflows FP32.
//
// Every thread carries a pair of cells in the two lanes of the paired FP32
// instructions: lane x works on parent t / new cell t of the tile, lane y on
// parent t + kThreadsMixed / new cell t + kThreadsMixed.  A tile has
// 2 kThreadsMixed parents and kTileMixed = 2 kThreadsMixed - 1 new cells.
// Parent records are stored interleaved ((slot t, slot t + kThreadsMixed) at
// index t) so that a new cell's two parents are one 64-bit shared-memory load
// each.
#pragma once

#include "wcc_convert.cuh"
#include "wcc_f2.cuh"
#include "wcc_ff.cuh"
#include "wcc_halfstep.cuh"

namespace wcc {

// Threads per CTA of the FP32-mixed kernels (two cells each).
#ifndef WCC_MIXED_THREADS
#define WCC_MIXED_THREADS 128
#endif
constexpr int kThreadsMixed = WCC_MIXED_THREADS;
constexpr int kTileMixed = 2 * kThreadsMixed - 1;

// Resident CTAs per SM the FP32-mixed kernels are compiled for (register
// budget 65536 / (kThreadsMixed * CTAs) per thread): the most that still
// compiles without spills (measured on GB300, Euler): 7 for P <= 2, 6 for
// P = 3, 5 for P = 4.  WCC_MIXED_MIN_CTAS overrides it for every P.
// Consecutive tiles per CTA of the single-grid kernel: 2 for P <= 2 (one
// CTA reduction for two tiles; measured faster), 1 for P >= 3 (measured
// slower with 2).
template <int P>
constexpr int mixed_tiles_per_cta() {
    return P <= 2 ? 2 : 1;
}

template <int P>
constexpr int mixed_min_ctas() {
#ifdef WCC_MIXED_MIN_CTAS
    return WCC_MIXED_MIN_CTAS;
#else
    return P <= 2 ? 7 : P == 3 ? 6 : 5;
#endif
}

// Where one tile reads and writes (one stage of one grid or batch instance).
struct TileIO {
    const float* in32;
    float* out32;
    long long pitch;
    long long n_old;
    long long n_new;
    long long first_new;
    int parity;
    int bc;
};

// ------------------------------------------------------ float-float pairs

struct ff2 {
    f2 hi, lo;
};

__device__ __forceinline__ ff2 two_sum2(f2 a, f2 b) {
    const f2 s = a + b;
    const f2 bb = s - a;
    const f2 e = (a - (s - bb)) + (b - bb);
    return ff2{s, e};
}

__device__ __forceinline__ ff2 fast_two_sum2(f2 a, f2 b) {
    const f2 s = a + b;
    const f2 e = b - (s - a);
    return ff2{s, e};
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
    const ff2 s = two_sum2(a.hi, b.hi);
    return fast_two_sum2(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, f2 b) {
    const ff2 s = two_sum2(a.hi, b);
    return fast_two_sum2(s.hi, s.lo + a.lo);
}

// a + b where b is itself only FP32-accurate: Fast2Sum in place of TwoSum.
// When |b| > |a.hi| the low bits lost are below ulp(b), within b's own error.
__device__ __forceinline__ ff2 ff2_add_fp32(ff2 a, f2 b) {
    const ff2 s = fast_two_sum2(a.hi, b);
    return fast_two_sum2(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff2 ff2_neg(ff2 a) { return ff2{-a.hi, -a.lo}; }
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return ff2_add(a, ff2_neg(b)); }
__device__ __forceinline__ ff2 ff2_scale(ff2 a, float pow2) { return ff2{a.hi * f2(pow2), a.lo * f2(pow2)}; }

__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
    const f2 p = a.hi * b.hi;
    const f2 e = fma(a.hi, b.hi, -p);
    return fast_two_sum2(p, fma(a.hi, b.lo, fma(a.lo, b.hi, e)));
}

// a / b for a normal b (a density): q1 = a.hi / b.hi, then the remainder
// a - b q1 -- its leading part a.hi - b.hi q1 is exact (q1 is close to the
// quotient, Sterbenz) and only needs FP32 accuracy -- divided by b.hi for
// the correction q2.  One reciprocal estimate serves both quotients.
__device__ __forceinline__ ff2 ff2_div(ff2 a, ff2 b) {
    const f2 rb = rcp_approx(b.hi);
    const f2 q1 = a.hi * rb;
    const f2 p = b.hi * q1;
    const f2 e = fma(b.hi, q1, -p);  // b.hi q1 = p + e exactly
    const f2 rem = (a.hi - p) + (a.lo - fma(b.lo, q1, e));
    return fast_two_sum2(q1, rem * rb);
}

// (a - b) rounded to a pair of floats, a and b close (Sterbenz on the hi parts)
__device__ __forceinline__ f2 ff2_diff(ff2 a, ff2 b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// Arithmetic on cell-average quantities: float-float (COMP = true, the
// FP32-mixed precision) or plain FP32 with the low parts kept at zero
// (COMP = false, the uncompensated FP32 precision used to measure what the
// compensation buys).
template <bool COMP>
struct FF {
    static __device__ __forceinline__ ff2 add(ff2 a, ff2 b) { return ff2_add(a, b); }
    static __device__ __forceinline__ ff2 add(ff2 a, f2 b) { return ff2_add_fp32(a, b); }
    static __device__ __forceinline__ ff2 sub(ff2 a, ff2 b) { return ff2_sub(a, b); }
    static __device__ __forceinline__ ff2 mul(ff2 a, ff2 b) { return ff2_mul(a, b); }
    static __device__ __forceinline__ ff2 div(ff2 a, ff2 b) { return ff2_div(a, b); }
    static __device__ __forceinline__ f2 diff(ff2 a, ff2 b) { return ff2_diff(a, b); }
};

template <>
struct FF<false> {
    static __device__ __forceinline__ ff2 mk(f2 h) { return ff2{h, f2(0.f)}; }
    static __device__ __forceinline__ ff2 add(ff2 a, ff2 b) { return mk(a.hi + b.hi); }
    static __device__ __forceinline__ ff2 add(ff2 a, f2 b) { return mk(a.hi + b); }
    static __device__ __forceinline__ ff2 sub(ff2 a, ff2 b) { return mk(a.hi - b.hi); }
    static __device__ __forceinline__ ff2 mul(ff2 a, ff2 b) { return mk(a.hi * b.hi); }
    static __device__ __forceinline__ ff2 div(ff2 a, ff2 b) { return mk(fdiv_fast(a.hi, b.hi)); }
    static __device__ __forceinline__ f2 diff(ff2 a, ff2 b) { return a.hi - b.hi; }
};

// Cell average minus centre value of the Taylor polynomial with coefficients
// c[1..P] (Eq. 1DPolynomial_Space integrated over the cell): sum over even
// k >= 2 of c_k / ((k + 1) 2^k).
template <int P>
__device__ __forceinline__ f2 average_minus_centre(const f2 (&c)[P + 1]) {
    f2 s(0.f);
    sfor<2, P + 1>([&](auto Ki) {
        constexpr int k = decltype(Ki)::value;
        if constexpr ((k & 1) == 0) s = fma(f2((float)(1.0 / ((k + 1.0) * cpow2(k)))), c[k], s);
    });
    return s;
}

template <int SYS, bool COMP>
__device__ __forceinline__ void flux_ff2(const ff2 (&u)[nvars(SYS)], const StepArgs& args, ff2 (&f)[nvars(SYS)]) {
    using A = FF<COMP>;
    if constexpr (SYS == ADVECTION) {
        f[0] = A::mul(u[0], ff2{f2(args.adv_hi), f2(COMP ? args.adv_lo : 0.f)});
    } else if constexpr (SYS == BURGERS) {
        f[0] = ff2_scale(A::mul(u[0], u[0]), 0.5f);
    } else {
        const ff2 w = A::div(u[1], u[0]);
        const ff2 q = A::mul(u[1], w);
        const ff2 p = A::mul(A::add(u[2], ff2_scale(q, -0.5f)), ff2{f2(args.g1_hi), f2(COMP ? args.g1_lo : 0.f)});
        f[0] = u[1];
        f[1] = A::add(q, p);
        f[2] = A::mul(A::add(u[2], p), w);
    }
}

// ------------------------------------------------------ limiter, paired

// Reciprocal estimate of each lane from the special-function unit (relative
// error about 2^-23), for normal or infinite inputs (0 gives +inf).
__device__ __forceinline__ f2 rcp_est(f2 a) {
    float rx, ry;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(a.v.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(a.v.y));
    return f2(rx, ry);
}

// The weights' denominators d = beta^2 + eps (beta + eps at P = 1) are
// formed scaled by 2^32, which is exact, with eps' = max(eps, 2^-149) so that
// d > 0.  The paper's eps = 1e-40 is subnormal in FP32; scaled, every d is a
// normal number, so each ratio a / d is one reciprocal estimate per lane and
// a paired multiply (for normal d the same value as a / d unscaled: the
// estimate of x 2^k is the estimate of x times 2^-k).
__device__ __forceinline__ f2 scaled_eps(const StepArgs& args) {
    return f2(fmaxf(args.eps_f, 1.4e-45f) * 4294967296.f);
}

// Normalised weights for P >= 2 (Eq. 1DHighOrderWeights), scale-free:
// w0 ~ 1 + (st/d0)^alpha, w_m ~ (st/d_m)^alpha with d = beta^2 + eps, all
// multiplied through by (d_min/st)^alpha, so every ratio is at most 1 (st = 0
// makes the first ratio +inf, clamped to 1e18).  w0 is formed as 1 - w1 - w2
// so that it is exactly 1 whenever the other two vanish.
__device__ __forceinline__ void weights_hi_f2(f2 b0, f2 b1, f2 b2, f2 st, const StepArgs& args, f2& w0, f2& w1,
                                              f2& w2) {
    const f2 eps = scaled_eps(args), s16(65536.f), s32(4294967296.f);
    const f2 c0 = b0 * s16, c1 = b1 * s16, c2 = b2 * s16;
    const f2 d0 = fma(c0, c0, eps), d1 = fma(c1, c1, eps), d2 = fma(c2, c2, eps);  // d 2^32
    const f2 dmin = fmin(d0, fmin(d1, d2));
    const f2 q0 = dmin * rcp_est(d0), q1 = dmin * rcp_est(d1), q2 = dmin * rcp_est(d2);
    const f2 z = fmin(dmin * rcp_est(st * s32), f2(1e18f));  // st = 0 gives +inf -> 1e18
    f2 h0, h1, h2;
    if (args.alpha_is_two) {
        h0 = fma(z, z, q0 * q0);
        h1 = q1 * q1;
        h2 = q2 * q2;
    } else {
        const float al = args.alpha_f;
        h0 = f2(__powf(z.x(), al) + __powf(q0.x(), al), __powf(z.y(), al) + __powf(q0.y(), al));
        h1 = f2(__powf(q1.x(), al), __powf(q1.y(), al));
        h2 = f2(__powf(q2.x(), al), __powf(q2.y(), al));
    }
    const f2 inv = rcp_est(h0 + h1 + h2);  // the sum is at least 1 (the ratio of d_min)
    w1 = h1 * inv;
    w2 = h2 * inv;
    w0 = f2(1.f) - (w1 + w2);
}

// Normalised weights for P = 1 (Eq. 1D2ndOrderWeights): w_m proportional to
// (1 / (beta_m + eps))^alpha, evaluated as ((beta_min + eps) / (beta_m + eps))^alpha <= 1.
__device__ __forceinline__ void weights_p1_f2(f2 b0, f2 b1, f2 b2, const StepArgs& args, f2& w0, f2& w1, f2& w2) {
    const f2 eps = scaled_eps(args), s32(4294967296.f);
    const f2 d0 = fma(b0, s32, eps), d1 = fma(b1, s32, eps), d2 = fma(b2, s32, eps);  // d 2^32
    const f2 dmin = fmin(d0, fmin(d1, d2));
    const f2 q0 = dmin * rcp_est(d0), q1 = dmin * rcp_est(d1), q2 = dmin * rcp_est(d2);
    f2 h0, h1, h2;
    if (args.alpha_is_two) {
        h0 = q0 * q0;
        h1 = q1 * q1;
        h2 = q2 * q2;
    } else {
        const float al = args.alpha_f;
        h0 = f2(__powf(q0.x(), al), __powf(q0.y(), al));
        h1 = f2(__powf(q1.x(), al), __powf(q1.y(), al));
        h2 = f2(__powf(q2.x(), al), __powf(q2.y(), al));
    }
    const f2 inv = rcp_est(h0 + h1 + h2);  // at least 1
    w1 = h1 * inv;
    w2 = h2 * inv;
    w0 = f2(1.f) - (w1 + w2);
}

// Limiter of Sec. 2.2 in deviation form, paired.  d[0] = u_0(centre) - ubar,
// d[1..P] = Taylor coefficients; dl = ubar - u_{i-1/2}, dr = u_{i+1/2} - ubar.
// On return d holds the same quantities of the limited polynomial.
template <int P>
__device__ __forceinline__ void limit_deviation_f2(f2 (&d)[P + 1], f2 dl, f2 dr, const StepArgs& args) {
    const f2 s1 = f2(2.f) * dl, s2 = f2(2.f) * dr;
    f2 b0(0.f);
    sfor<1, P + 1>([&](auto Ji) {
        constexpr int j = decltype(Ji)::value;
        f2 row(0.f);
        sfor<j, P + 1>([&](auto Li) {
            constexpr int l = decltype(Li)::value;
            constexpr double cjl = (l == j ? 1.0 : 2.0) * csmooth(j, l);
            if constexpr (cjl != 0.0) row = fma(f2((float)cjl), d[l], row);
        });
        b0 = fma(row, d[j], b0);
    });
    const f2 b1 = s1 * s1, b2 = s2 * s2;
    f2 w0, w1, w2;
    if constexpr (P == 1) {
        weights_p1_f2(b0, b1, b2, args, w0, w1, w2);
    } else {
        f2 up = d[0], um = d[0];
        sfor<1, P + 1>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            up = fma(f2((float)chalf(k, false)), d[k], up);
            um = fma(f2((float)chalf(k, true)), d[k], um);
        });
        const f2 rr = up - dr;
        const f2 rl = um + dl;
        const f2 sigma = fma(rr, rr, rl * rl);
        const f2 tp = f2((float)cfact(P)) * d[P];
        weights_hi_f2(b0, b1, b2, sigma * (tp * tp), args, w0, w1, w2);
    }
    d[0] *= w0;
    d[1] = fma(w0, d[1], fma(w1, s1, w2 * s2));
    sfor<2, P + 1>([&](auto Ki) { d[decltype(Ki)::value] *= w0; });
}

// ------------------------------------------------------ the paired tile

template <int SYS, int P>
constexpr int mixed2_smem_float2() {
    return nvars(SYS) * (5 + P) * (kThreadsMixed + 1);
}

// One tile of the FP32-mixed half-step, two cells per thread: parents
// io.first_new + s - parity for slots s = 0..2 kThreadsMixed - 1, new cells
// io.first_new + c for c = 0..kTileMixed - 1.  rec: mixed2_smem_float2 float2
// of shared memory.  Returns the larger of the thread's two cell speeds
// (cells outside the stage count as 0) and error bits; the caller
// synchronises the block before rec is written again.
template <int SYS, int P, bool COMP, bool PARK = (P >= 3)>
__device__ __forceinline__ void mixed_tile2(const TileIO& io, const ff lam, const StepArgs& args, float2* rec,
                                            float& speed, unsigned& err) {
    using A = FF<COMP>;
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NP = P + 2;
    constexpr int RV = 5 + P;
    constexpr int W = kThreadsMixed + 1;  // row width of rec in float2
    const int t = threadIdx.x;
    const long long first_new = io.first_new;
    const ff2 lam2{f2(lam.hi), f2(COMP ? lam.lo : 0.f)};

    // ---- phase 1: parent records of slots t (lane x) and t + kThreadsMixed (lane y)
    {
        const long long base = first_new + t - (io.parity ? 1 : 0);
        const long long pa = parent_index(base, io.n_old, io.bc);
        const long long pb = parent_index(base + kThreadsMixed, io.n_old, io.bc);
        // record row `row` of variable v for this thread's slots; slot
        // kThreadsMixed (lane y of thread 0) is also the right parent of new
        // cell kThreadsMixed - 1 (lane x of the last thread), whose y lane
        // repeats the value so that the unused lane sees real data
        auto put = [&](int v, int row, f2 x) {
            float2* r = rec + v * RV * W + row * W;
            r[t] = x.v;
            if (t == 0) r[kThreadsMixed] = make_float2(x.y(), x.y());
        };
        auto get = [&](int v, int row) { return f2(rec[v * RV * W + row * W + t]); };
        // With PARK (the default for P >= 3), ubar and lam f(u_0) wait in
        // their record rows (0-1 and 2-3) while the Cauchy-Kovalewski table
        // holds the registers; for lower P alone they fit in registers, which
        // is faster.
        constexpr bool kPark = PARK;
        f2 c[NV][K];
        ff2 ub_r[NV], lf_r[NV];
        {
            ff2 u0[NV];
            sfor<0, NV>([&](auto V) {
                constexpr int v = decltype(V)::value;
                const float* p0 = io.in32 + (long long)(v * NP + 0) * io.pitch;
                const float* p1 = io.in32 + (long long)(v * NP + 1) * io.pitch;
                ff2 ub;
                ub.hi = f2(__ldg(p0 + pa), __ldg(p0 + pb));
                ub.lo = COMP ? f2(__ldg(p1 + pa), __ldg(p1 + pb)) : f2(0.f);
                sfor<1, K>([&](auto Ki) {
                    constexpr int k = decltype(Ki)::value;
                    const float* pk = io.in32 + (long long)(v * NP + k + 1) * io.pitch;
                    c[v][k] = f2(__ldg(pk + pa), __ldg(pk + pb));
                });
                u0[v] = A::add(ub, -average_minus_centre<P>(c[v]));
                c[v][0] = u0[v].hi;
                if constexpr (kPark) {
                    put(v, 0, ub.hi);
                    if constexpr (COMP) put(v, 1, ub.lo);
                } else {
                    ub_r[v] = ub;
                }
            });
            ff2 f0[NV];
            flux_ff2<SYS, COMP>(u0, args, f0);
            sfor<0, NV>([&](auto V) {
                constexpr int v = decltype(V)::value;
                const ff2 lf = A::mul(f0[v], lam2);
                if constexpr (kPark) {
                    put(v, 2, lf.hi);
                    if constexpr (COMP) put(v, 3, lf.lo);
                } else {
                    lf_r[v] = lf;
                }
            });
        }
        f2 X[NV][K][K], F0[NV][K];
        ck_table<SYS, P, f2>(c, lam2.hi, args, X, F0);
        // Record of the parent (Eqs. Cal1DFlux, SubEq:1DCellAVGR/L,
        // SubEq:Cal_1D_Derivatives_4): its cell average ubar and
        //   A   = ubar / 2 + g,  g = lam fbar + dodd / 2, the part of ubar that
        //         goes to the new cell on its right (float-float; the new cell
        //         on its left gets B = ubar - A, so the scheme stays
        //         conservative to float-float rounding),
        //   dev = v_0 - ubar, the centre value at the new time level minus the
        //         cell average,
        //   and the higher vertex coefficients sum_m X[k][m], k >= 1.
        // g is lam f(u_0) in float-float plus the FP32 rest
        // h = lam (fbar - f(u_0)) + dodd / 2.
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            f2 fhigh(0.f);
            sfor<1, K>([&](auto Bi) {
                constexpr int b = decltype(Bi)::value;
                fhigh = fma(f2((float)(1.0 / (b + 1.0))), F0[v][b], fhigh);
            });
            f2 dodd(0.f);
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                if constexpr (k & 1) dodd = fma(f2((float)(1.0 / ((k + 1.0) * cpow2(k)))), c[v][k], dodd);
            });
            const f2 h = fma(lam2.hi, fhigh, f2(0.5f) * dodd);
            ff2 ub, lf;
            if constexpr (kPark) {
                ub = ff2{get(v, 0), COMP ? get(v, 1) : f2(0.f)};
                lf = ff2{get(v, 2), COMP ? get(v, 3) : f2(0.f)};
            } else {
                ub = ub_r[v];
                lf = lf_r[v];
                put(v, 0, ub.hi);
                if constexpr (COMP) put(v, 1, ub.lo);
            }
            const ff2 Ac = A::add(ff2_scale(ub, 0.5f), A::add(lf, h));
            put(v, 2, Ac.hi);
            if constexpr (COMP) put(v, 3, Ac.lo);
            f2 vt0(0.f);
            sfor<1, K>([&](auto Mi) { vt0 += X[v][0][decltype(Mi)::value]; });
            put(v, 4, vt0 - average_minus_centre<P>(c[v]));
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                f2 s = X[v][k][0];
                sfor<1, K - k>([&](auto Mi) { s += X[v][k][decltype(Mi)::value]; });
                put(v, 4 + k, s);
            });
        });
    }
    __syncthreads();

    // ---- phase 2: new cells t (lane x) and t + kThreadsMixed (lane y)
    const long long ia = first_new + t;
    const long long ib = first_new + kThreadsMixed + t;
    const bool va = ia < io.n_new;
    const bool vb = (t < kThreadsMixed - 1) && ib < io.n_new;
    ff2 ubn[NV];
    f2 d[NV][K], dl[NV], dr[NV];
    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        const float2* r = rec + v * RV * W;
        const f2 zero(0.f);
        const ff2 uL{f2(r[0 * W + t]), COMP ? f2(r[1 * W + t]) : zero};
        const ff2 uR{f2(r[0 * W + t + 1]), COMP ? f2(r[1 * W + t + 1]) : zero};
        const ff2 AL{f2(r[2 * W + t]), COMP ? f2(r[3 * W + t]) : zero};
        const ff2 AR{f2(r[2 * W + t + 1]), COMP ? f2(r[3 * W + t + 1]) : zero};
        const f2 eL(r[4 * W + t]), eR(r[4 * W + t + 1]);
        ubn[v] = A::add(AL, A::sub(uR, AR));  // Eq. SubEq:1DIntegral: A_L + B_R
        // vertex values v_L = ubar_L + dev_L, v_R = ubar_R + dev_R, taken
        // relative to the new average through differences of close numbers
        dl[v] = A::diff(ubn[v], uL) - eL;  // ubar_new - v_L
        dr[v] = A::diff(uR, ubn[v]) + eR;  // v_R - ubar_new
        f2 vL[K], vR[K];
        vL[0] = f2(0.f);
        vR[0] = A::diff(uR, uL) + (eR - eL);
        sfor<1, K>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            vL[k] = f2(r[(4 + k) * W + t]);
            vR[k] = f2(r[(4 + k) * W + t + 1]);
        });
        derivatives_and_point_value<P, f2>(f2(0.f), vL, vR, d[v]);
    });

    if (args.limiter) {
        if constexpr (NV == 1) {
            limit_deviation_f2<P>(d[0], dl[0], dr[0], args);
        } else {
            f2 ubf[3] = {ubn[0].hi, ubn[1].hi, ubn[2].hi};
            EulerChar<f2> E;
            if (!euler_char<f2>(ubf, f2(args.gamma_f), E)) err |= ERR_POSITIVITY;
            f2 cd[3][K], cdl[3], cdr[3];
            E.left(dl[0], dl[1], dl[2], cdl);
            E.left(dr[0], dr[1], dr[2], cdr);
            sfor<0, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                f2 w[3];
                E.left(d[0][k], d[1][k], d[2][k], w);
                cd[0][k] = w[0];
                cd[1][k] = w[1];
                cd[2][k] = w[2];
            });
            sfor<0, 3>([&](auto Ii) {
                constexpr int rr = decltype(Ii)::value;
                limit_deviation_f2<P>(cd[rr], cdl[rr], cdr[rr], args);
            });
            sfor<0, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                E.right(cd[0][k], cd[1][k], cd[2][k], d[0][k], d[1][k], d[2][k]);
            });
        }
    }

    f2 u0n[NV];
    f2 check(0.f);  // NaN / Inf in any stored value reaches this sum
    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        check += ubn[v].hi;
        float* o0 = io.out32 + (long long)(v * NP + 0) * io.pitch;
        float* o1 = io.out32 + (long long)(v * NP + 1) * io.pitch;
        if (va) {
            __stcs(o0 + ia, ubn[v].hi.x());
            __stcs(o1 + ia, ubn[v].lo.x());
        }
        if (vb) {
            __stcs(o0 + ib, ubn[v].hi.y());
            __stcs(o1 + ib, ubn[v].lo.y());
        }
        sfor<1, K>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            check += d[v][k];
            float* ok = io.out32 + (long long)(v * NP + k + 1) * io.pitch;
            if (va) __stcs(ok + ia, d[v][k].x());
            if (vb) __stcs(ok + ib, d[v][k].y());
        });
        u0n[v] = ubn[v].hi + d[v][0];
    });
    if ((va && not_finite(check.x())) || (vb && not_finite(check.y()))) err |= ERR_NONFINITE;
    const f2 sp = wave_speed<SYS, f2>(u0n, args, err);
    speed = fmaxf(va ? sp.x() : 0.f, vb ? sp.y() : 0.f);
}

template <int SYS, int P, bool COMP = true>
__global__ void __launch_bounds__(kThreadsMixed, mixed_min_ctas<P>()) halfstep_mixed2(const StepArgs args) {
    __shared__ float2 rec[mixed2_smem_float2<SYS, P>()];
    constexpr int TPC = mixed_tiles_per_cta<P>();
    const StepSize z = step_size(args);
    float speed = 0.f;
    unsigned err = 0u;
    if constexpr (TPC == 1) {
        const TileIO io{args.in32, args.out32, args.pitch, args.n_old, args.n_new,
                        (long long)blockIdx.x * kTileMixed, args.parity, args.bc};
        mixed_tile2<SYS, P, COMP>(io, ff_make(z.lam_hi, z.lam_lo), args, rec, speed, err);
    } else {
        const long long ntiles = (args.n_new + kTileMixed - 1) / kTileMixed;
        for (int r = 0; r < TPC; ++r) {
            const long long tile = (long long)blockIdx.x * TPC + r;
            if (tile >= ntiles) break;
            if (r) __syncthreads();  // the previous tile's records are read
            const TileIO io{args.in32, args.out32, args.pitch, args.n_old, args.n_new,
                            tile * kTileMixed, args.parity, args.bc};
            float sp = 0.f;
            mixed_tile2<SYS, P, COMP>(io, ff_make(z.lam_hi, z.lam_lo), args, rec, sp, err);
            speed = fmaxf(speed, sp);
        }
    }
    finish_halfstep<float, kThreadsMixed>(speed, err, z.dt, args);
}

// Set-up of an FP32-mixed stage in one pass: the host-layout DOFs (already in
// device memory) are converted tile by tile through shared memory with the
// conversions of wcc_convert.cuh (plain FP32 keeps only the rounded
// average), and the largest characteristic speed at the centre values of the
// stored planes goes to st->amax_bits[slot] (zero beforehand).
constexpr int kLoadCells = 128;  // cells per tile = threads per CTA

template <int SYS, int P>
__global__ void __launch_bounds__(kLoadCells) load_stage_mixed(const double* __restrict__ aos, long long n,
                                                               long long pitch, float* __restrict__ planes,
                                                               int keep_lo, StepArgs args, int slot) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NP = P + 2;
    constexpr int ROW = NV * K;
    __shared__ unsigned long long sm[kLoadCells * ROW];  // DOFs as bit patterns
    float m = 0.f;  // the largest float speed, converted once at the end
    unsigned err = 0u;
    for (long long c0 = (long long)blockIdx.x * kLoadCells; c0 < n; c0 += (long long)gridDim.x * kLoadCells) {
        const int cnt = (int)min((long long)kLoadCells, n - c0);
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(aos) + c0 * ROW;
        for (int i = threadIdx.x; i < cnt * ROW; i += kLoadCells) sm[i] = src[i];
        __syncthreads();
        const int c = threadIdx.x;
        if (c < cnt) {
            float u0[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                float e[K];
                const ff u = host_to_mixed<K>(sm + c * ROW + v * K, e);
                const float lo = keep_lo ? u.lo : 0.f;
                float* pl = planes + (long long)(v * NP) * pitch + c0 + c;
                pl[0] = u.hi;
                pl[pitch] = lo;
#pragma unroll
                for (int k = 1; k < K; ++k) pl[(long long)(k + 1) * pitch] = e[k];
                // centre value of the stored cell: average minus the even terms
                float corr = 0.f;
#pragma unroll
                for (int k = 2; k <= P; k += 2) corr += e[k] / (float)((k + 1) * (1 << k));
                u0[v] = (u.hi + lo) - corr;
            }
            float sp = wave_speed<SYS, float>(u0, args, err);
            if (sp != sp) {
                sp = INFINITY;
                err |= ERR_NONFINITE;
            }
            m = fmaxf(m, sp);
        }
        __syncthreads();
    }
    m = warp_max<float>(m);
    if ((threadIdx.x & 31) == 0 && m > 0.f)
        atomicMax(&args.st->amax_bits[slot], (unsigned long long)__double_as_longlong((double)m));
    if (err) atomicOr(&args.st->err, err);
}

}  // namespace wcc
