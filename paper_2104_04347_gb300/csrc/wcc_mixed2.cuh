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
// P = 3, 5 for P = 4; 4 (128 registers) for P = 5, 6.  WCC_MIXED_MIN_CTAS
// overrides it for every P.
// Consecutive tiles per CTA of the single-grid kernel: 2 for P <= 2 (one
// CTA reduction for two tiles; measured faster), 1 for P >= 3 (measured
// slower with 2).
__host__ __device__ constexpr int mixed_default_tiles(int P) { return P <= 2 ? 2 : 1; }

template <int P>
constexpr int mixed_tiles_per_cta() {
    return mixed_default_tiles(P);
}

template <int P>
constexpr int mixed_min_ctas() {
#ifdef WCC_MIXED_MIN_CTAS
    return WCC_MIXED_MIN_CTAS;
#else
    return P <= 2 ? 7 : P == 3 ? 6 : P == 4 ? 5 : 4;
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

// a + b where b is itself only FP32-accurate: Fast2Sum in place of TwoSum.
// When |b| > |a.hi| the low bits lost are below ulp(b), within b's own error.
__device__ __forceinline__ ff2 ff2_add_fp32(ff2 a, f2 b) {
    const ff2 s = fast_two_sum2(a.hi, b);
    return fast_two_sum2(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff2 ff2_scale(ff2 a, float pow2) { return ff2{a.hi * f2(pow2), a.lo * f2(pow2)}; }

// (a - b) rounded to a pair of floats, a and b close (Sterbenz on the hi parts)
__device__ __forceinline__ f2 ff2_diff(ff2 a, ff2 b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// Sums, products and quotients without a closing renormalisation, for
// results that only feed further float-float arithmetic: (hi, lo) with lo a
// few ulp of hi is as exact a representation of the value, and every
// operation here reads both parts (a product takes hi * hi exactly and the lo
// cross terms).
__device__ __forceinline__ ff2 ff2_add_u(ff2 a, ff2 b) {
    const ff2 s = two_sum2(a.hi, b.hi);
    return ff2{s.hi, s.lo + (a.lo + b.lo)};
}
__device__ __forceinline__ ff2 ff2_add_fp32_u(ff2 a, f2 b) {
    const ff2 s = fast_two_sum2(a.hi, b);
    return ff2{s.hi, s.lo + a.lo};
}
__device__ __forceinline__ ff2 ff2_mul_u(ff2 a, ff2 b) {
    const f2 p = a.hi * b.hi;
    const f2 e = fma(a.hi, b.hi, -p);
    return ff2{p, fma(a.hi, b.lo, fma(a.lo, b.hi, e))};
}
// a / b for a normal b (a density): q1 = a.hi / b.hi, then the remainder
// a - b q1 -- its leading part a.hi - b.hi q1 is exact (q1 is close to the
// quotient, Sterbenz) and only needs FP32 accuracy -- divided by b.hi for
// the correction q2.  One reciprocal estimate serves both quotients.
__device__ __forceinline__ ff2 ff2_div_u(ff2 a, ff2 b) {
    const f2 rb = rcp_approx(b.hi);
    const f2 q1 = a.hi * rb;
    const f2 p = b.hi * q1;
    const f2 e = fma(b.hi, q1, -p);  // b.hi q1 = p + e exactly
    const f2 rem = (a.hi - p) + (a.lo - fma(b.lo, q1, e));
    return ff2{q1, rem * rb};
}
// a / 2 + b + c for b's FP32-accurate correction c (Fast2Sum on b + c as in
// ff2_add_fp32), with one renormalisation at the end
__device__ __forceinline__ ff2 ff2_half_plus(ff2 a, ff2 b, f2 c) {
    const ff2 x = fast_two_sum2(b.hi, c);
    const ff2 y = two_sum2(a.hi * f2(0.5f), x.hi);
    return fast_two_sum2(y.hi, ((a.lo * f2(0.5f) + b.lo) + x.lo) + y.lo);
}
// a + (b - c) with one renormalisation at the end
__device__ __forceinline__ ff2 ff2_add_diff(ff2 a, ff2 b, ff2 c) {
    const ff2 x = two_sum2(b.hi, -c.hi);
    const ff2 y = two_sum2(a.hi, x.hi);
    return fast_two_sum2(y.hi, ((b.lo - c.lo) + a.lo) + (x.lo + y.lo));
}

// Arithmetic on cell-average quantities: float-float (COMP = true, the
// FP32-mixed precision) or plain FP32 with the low parts kept at zero
// (COMP = false, the uncompensated FP32 precision used to measure what the
// compensation buys).
template <bool COMP>
struct FF {
    static __device__ __forceinline__ ff2 add(ff2 a, f2 b) { return ff2_add_fp32(a, b); }
    static __device__ __forceinline__ f2 diff(ff2 a, ff2 b) { return ff2_diff(a, b); }
    static __device__ __forceinline__ ff2 add_u(ff2 a, ff2 b) { return ff2_add_u(a, b); }
    static __device__ __forceinline__ ff2 add_u(ff2 a, f2 b) { return ff2_add_fp32_u(a, b); }
    static __device__ __forceinline__ ff2 mul_u(ff2 a, ff2 b) { return ff2_mul_u(a, b); }
    static __device__ __forceinline__ ff2 div_u(ff2 a, ff2 b) { return ff2_div_u(a, b); }
    static __device__ __forceinline__ ff2 half_plus(ff2 a, ff2 b, f2 c) { return ff2_half_plus(a, b, c); }
    static __device__ __forceinline__ ff2 add_diff(ff2 a, ff2 b, ff2 c) { return ff2_add_diff(a, b, c); }
};

template <>
struct FF<false> {
    static __device__ __forceinline__ ff2 mk(f2 h) { return ff2{h, f2(0.f)}; }
    static __device__ __forceinline__ ff2 add(ff2 a, ff2 b) { return mk(a.hi + b.hi); }
    static __device__ __forceinline__ ff2 add(ff2 a, f2 b) { return mk(a.hi + b); }
    static __device__ __forceinline__ ff2 mul(ff2 a, ff2 b) { return mk(a.hi * b.hi); }
    static __device__ __forceinline__ ff2 div(ff2 a, ff2 b) { return mk(fdiv_fast(a.hi, b.hi)); }
    static __device__ __forceinline__ f2 diff(ff2 a, ff2 b) { return a.hi - b.hi; }
    static __device__ __forceinline__ ff2 add_u(ff2 a, ff2 b) { return add(a, b); }
    static __device__ __forceinline__ ff2 add_u(ff2 a, f2 b) { return add(a, b); }
    static __device__ __forceinline__ ff2 mul_u(ff2 a, ff2 b) { return mul(a, b); }
    static __device__ __forceinline__ ff2 div_u(ff2 a, ff2 b) { return div(a, b); }
    static __device__ __forceinline__ ff2 half_plus(ff2 a, ff2 b, f2 c) { return mk(a.hi * f2(0.5f) + (b.hi + c)); }
    static __device__ __forceinline__ ff2 add_diff(ff2 a, ff2 b, ff2 c) { return mk(a.hi + (b.hi - c.hi)); }
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
        f[0] = A::mul_u(u[0], ff2{f2(args.adv_hi), f2(COMP ? args.adv_lo : 0.f)});
    } else if constexpr (SYS == BURGERS) {
        f[0] = ff2_scale(A::mul_u(u[0], u[0]), 0.5f);
    } else {
        // every result feeds float-float arithmetic again (lam f below):
        // no renormalisation in between
        const ff2 w = A::div_u(u[1], u[0]);
        const ff2 q = A::mul_u(u[1], w);
        const ff2 p = A::mul_u(A::add_u(u[2], ff2_scale(q, -0.5f)), ff2{f2(args.g1_hi), f2(COMP ? args.g1_lo : 0.f)});
        f[0] = u[1];
        f[1] = A::add_u(q, p);
        f[2] = A::mul_u(A::add_u(u[2], p), w);
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

// The tile is built from four steps that the single half-step runs in a row
// (mixed_tile2) and the two-half-step kernel twice (halfstep_mixed2_tb2):
//   mixed_load_parents    the parents' stored values from a stage in global memory,
//   mixed_parent_records  phase 1: each parent's record into rec,
//   mixed_new_cells       phase 2: the new cells from neighbouring records,
//   mixed_store           the new cells into a stage in global memory.
// Parents are slots s = 0..2 kThreadsMixed - 1 (lane x: s = t, lane y:
// s = t + kThreadsMixed); new cell c is built from slots c and c + 1.

// Values of parent slots t and t + kThreadsMixed (stage index
// io.first_new + s - parity, through the boundary rule): the cell average
// ub (float-float) and the Taylor coefficients c[v][1..P] (c[v][0] is left
// for mixed_parent_records).
template <int SYS, int P, bool COMP>
__device__ __forceinline__ void mixed_load_parents(const TileIO& io, ff2 (&ub)[nvars(SYS)],
                                                   f2 (&c)[nvars(SYS)][P + 1]) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NP = P + 2;
    const int t = threadIdx.x;
    const long long base = io.first_new + t - (io.parity ? 1 : 0);
    const long long pa = parent_index(base, io.n_old, io.bc);
    const long long pb = parent_index(base + kThreadsMixed, io.n_old, io.bc);
    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        const float* p0 = io.in32 + (long long)(v * NP + 0) * io.pitch;
        const float* p1 = io.in32 + (long long)(v * NP + 1) * io.pitch;
        ub[v].hi = f2(__ldg(p0 + pa), __ldg(p0 + pb));
        ub[v].lo = COMP ? f2(__ldg(p1 + pa), __ldg(p1 + pb)) : f2(0.f);
        sfor<1, K>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            const float* pk = io.in32 + (long long)(v * NP + k + 1) * io.pitch;
            c[v][k] = f2(__ldg(pk + pa), __ldg(pk + pb));
        });
    });
}

// Phase 1: the records of this thread's two parents (cell averages ub,
// coefficients c[v][1..P]; c[v][0] is overwritten) into rec.  The caller
// synchronises the block before reading rec.
template <int SYS, int P, bool COMP, bool PARK = (P >= 3)>
__device__ __forceinline__ void mixed_parent_records(const ff2 (&ub_in)[nvars(SYS)], f2 (&c)[nvars(SYS)][P + 1],
                                                     const ff2 lam2, const StepArgs& args, float2* rec) {
    using A = FF<COMP>;
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int RV = 5 + P;
    constexpr int W = kThreadsMixed + 1;  // row width of rec in float2
    const int t = threadIdx.x;
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
    ff2 ub_r[NV], lf_r[NV];
    {
        ff2 u0[NV];
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            const ff2 ub = ub_in[v];
            // normalised: its high part is the float point value of the
            // Cauchy-Kovalewski table
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
            const ff2 lf = A::mul_u(f0[v], lam2);
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
        const ff2 Ac = A::half_plus(ub, lf, h);
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

// Phase 2: new cells t (lane x) and t + kThreadsMixed (lane y) from the
// records of slots (t, t + 1) and (t + kThreadsMixed, t + kThreadsMixed + 1):
// the cell average ubn (float-float), the point value minus the average
// d[v][0] and the coefficients d[v][1..P] of the limited polynomial.
template <int SYS, int P, bool COMP>
__device__ __forceinline__ void mixed_new_cells(const float2* rec, const StepArgs& args, ff2 (&ubn)[nvars(SYS)],
                                                f2 (&d)[nvars(SYS)][P + 1], unsigned& err) {
    using A = FF<COMP>;
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int RV = 5 + P;
    constexpr int W = kThreadsMixed + 1;
    const int t = threadIdx.x;
    f2 dl[NV], dr[NV];
    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        const float2* r = rec + v * RV * W;
        const f2 zero(0.f);
        const ff2 uL{f2(r[0 * W + t]), COMP ? f2(r[1 * W + t]) : zero};
        const ff2 uR{f2(r[0 * W + t + 1]), COMP ? f2(r[1 * W + t + 1]) : zero};
        const ff2 AL{f2(r[2 * W + t]), COMP ? f2(r[3 * W + t]) : zero};
        const ff2 AR{f2(r[2 * W + t + 1]), COMP ? f2(r[3 * W + t + 1]) : zero};
        const f2 eL(r[4 * W + t]), eR(r[4 * W + t + 1]);
        ubn[v] = A::add_diff(AL, uR, AR);  // Eq. SubEq:1DIntegral: A_L + B_R
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
            // the point value less the average is minus the even
            // correction of the coefficients k >= 2 (the limiter keeps the
            // average), a linear map that the projections commute with: it
            // is formed on each side instead of being projected
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                f2 w[3];
                E.left(d[0][k], d[1][k], d[2][k], w);
                cd[0][k] = w[0];
                cd[1][k] = w[1];
                cd[2][k] = w[2];
            });
            sfor<0, 3>([&](auto Ii) {
                constexpr int rr = decltype(Ii)::value;
                cd[rr][0] = -average_minus_centre<P>(cd[rr]);
                limit_deviation_f2<P>(cd[rr], cdl[rr], cdr[rr], args);
            });
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                E.right(cd[0][k], cd[1][k], cd[2][k], d[0][k], d[1][k], d[2][k]);
            });
            sfor<0, 3>([&](auto Vi) {
                constexpr int v = decltype(Vi)::value;
                d[v][0] = -average_minus_centre<P>(d[v]);
            });
        }
    }
}

// Largest characteristic speed at the centre values ubn + d[v][0] of the
// thread's two new cells, counting a lane only if it is valid.
template <int SYS>
__device__ __forceinline__ float mixed_cell_speed(const ff2 (&ubn)[nvars(SYS)], const f2 (&d0)[nvars(SYS)],
                                                  bool va, bool vb, const StepArgs& args, unsigned& err) {
    f2 u0n[nvars(SYS)];
    sfor<0, nvars(SYS)>([&](auto V) { u0n[decltype(V)::value] = ubn[decltype(V)::value].hi + d0[decltype(V)::value]; });
    const f2 sp = wave_speed<SYS, f2>(u0n, args, err);
    return fmaxf(va ? sp.x() : 0.f, vb ? sp.y() : 0.f);
}

// New cells io.first_new + t (lane x, if va) and io.first_new + t +
// kThreadsMixed (lane y, if vb) into the stage io.out32; returns the larger
// of their speeds.
template <int SYS, int P>
__device__ __forceinline__ float mixed_store(const TileIO& io, const ff2 (&ubn)[nvars(SYS)],
                                             const f2 (&d)[nvars(SYS)][P + 1], bool va, bool vb,
                                             const StepArgs& args, unsigned& err) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NP = P + 2;
    const long long ia = io.first_new + threadIdx.x;
    const long long ib = ia + kThreadsMixed;
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
    return fmaxf(va ? sp.x() : 0.f, vb ? sp.y() : 0.f);
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
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    const int t = threadIdx.x;
    const ff2 lam2{f2(lam.hi), f2(COMP ? lam.lo : 0.f)};
    {
        ff2 ub[NV];
        f2 c[NV][K];
        mixed_load_parents<SYS, P, COMP>(io, ub, c);
        mixed_parent_records<SYS, P, COMP, PARK>(ub, c, lam2, args, rec);
    }
    __syncthreads();
    ff2 ubn[NV];
    f2 d[NV][K];
    mixed_new_cells<SYS, P, COMP>(rec, args, ubn, d, err);
    const long long ia = io.first_new + t;
    const bool va = ia < io.n_new;
    const bool vb = (t < kThreadsMixed - 1) && ia + kThreadsMixed < io.n_new;
    speed = mixed_store<SYS, P>(io, ubn, d, va, vb, args, err);
}

// One half-step over a stage; each CTA handles TPC consecutive tiles
// (kTileMixed new cells each), one CTA reduction for all of them.
template <int SYS, int P, bool COMP = true, int TPC = mixed_tiles_per_cta<P>()>
__global__ void __launch_bounds__(kThreadsMixed, mixed_min_ctas<P>()) halfstep_mixed2(const StepArgs args) {
    __shared__ float2 rec[mixed2_smem_float2<SYS, P>()];
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

// ------------------------------------------------------ two half-steps per launch

// Final cells of a two-half-step tile: 2 kThreadsMixed parents give
// 2 kThreadsMixed - 1 intermediate cells and 2 kThreadsMixed - 2 final ones.
constexpr int kTileTB = 2 * kThreadsMixed - 2;

// Where one pair's bookkeeping goes: the device state of the problem (a
// single grid, or one batch instance), its dt history, its mesh width, the
// CFL numbers, and -- batches only -- the copy of the state taken before the
// pair and the batch's refusal flag.
struct PairBook {
    DevState* st;
    double* hist;
    long long hist_cap;
    long long ctas;     // CTAs (tiles) that count towards this state
    double dx;
    double cfl;
    double nu_max;      // the second half-step's largest CFL number
    int cfl_mode;
    int parity;
    DevState* backup;   // batches: the state before the pair, or nullptr
    unsigned* refused;  // batches: set to 1 when this state refuses the pair, or nullptr
};

// Bookkeeping of a two-half-step launch after the last CTA of a problem
// finished (one thread): the pair is taken when the realised CFL number of
// its second half-step, dt a_mid / dx with a_mid the bound of the
// intermediate stage, is at most nu_max; then dt is recorded twice, t
// advances by two steps and the next launch's dt comes from the final
// stage's bound, as in finalize_state.  Otherwise the refusal is flagged
// (ERR_CFL in the state, and the batch's flag) and the state (t, step, the
// bounds of the input stage and the prepared dt) is left as it was before
// the launch, so that the caller can take the two half-steps one by one
// from the input stage, which the launch did not overwrite.
__device__ __forceinline__ void finalize_pair(const PairBook& bk, double dt) {
    DevState* st = bk.st;
    const int parity = bk.parity;
    const float fmid = __uint_as_float(st->amax_f32[parity ^ 1]);
    const float ffin = __uint_as_float(st->amax_f32_tb);
    st->amax_f32[parity ^ 1] = 0u;
    st->amax_f32_tb = 0u;
    st->blocks_done = 0u;
    if (bk.backup) *bk.backup = *st;
    const double nu2 = dt * (double)fmid / bk.dx;
    if (!(nu2 <= bk.nu_max)) {
        st->err |= ERR_CFL;
        if (bk.refused) atomicExch(bk.refused, 1u);
        __threadfence();
        return;
    }
    if (nu2 > st->tb_nu2_max) st->tb_nu2_max = nu2;
    st->amax_bits[parity ^ 1] = (unsigned long long)__double_as_longlong((double)fmid);
    st->amax_bits[parity] = (unsigned long long)__double_as_longlong((double)ffin);
    const long long k = st->step;
    if (k < bk.hist_cap) bk.hist[k] = dt;
    if (k + 1 < bk.hist_cap) bk.hist[k + 1] = dt;
    st->step = k + 2;
    st->t = (st->t + dt) + dt;
    if (not_finite(dt)) st->err |= ERR_NONFINITE;
    if (bk.cfl_mode) {
        const double ndt = bk.cfl * bk.dx / (double)ffin;
        st->next_dt = ndt;
        st->next_lam = ndt / bk.dx;
        split_to_floats(st->next_lam, st->next_lam_hi, st->next_lam_lo);
        st->next_cfl = bk.cfl;
    } else {
        st->next_cfl = 0.0;
    }
    __threadfence();
}

// Block maxima of the intermediate and final speeds, one atomic each per
// CTA into the problem's state, then the CTA count; the CTA that completes
// bk.ctas runs finalize_pair.  Synchronises the block.
__device__ __forceinline__ void finish_pair(float mid, float fin, unsigned err, double dt, const PairBook& bk) {
    __shared__ float s_mid[kThreadsMixed / 32], s_fin[kThreadsMixed / 32];
    __shared__ unsigned s_err[kThreadsMixed / 32];
    if (mid != mid) {
        mid = INFINITY;
        err |= ERR_NONFINITE;
    }
    if (fin != fin) {
        fin = INFINITY;
        err |= ERR_NONFINITE;
    }
    mid = warp_max<float>(mid);
    fin = warp_max<float>(fin);
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
        s_mid[threadIdx.x >> 5] = mid;
        s_fin[threadIdx.x >> 5] = fin;
        s_err[threadIdx.x >> 5] = err;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = s_mid[0], f = s_fin[0];
        unsigned e = s_err[0];
#pragma unroll
        for (int w = 1; w < kThreadsMixed / 32; ++w) {
            m = fmaxf(m, s_mid[w]);
            f = fmaxf(f, s_fin[w]);
            e |= s_err[w];
        }
        DevState* st = bk.st;
        if (m > 0.f) atomicMax(&st->amax_f32[bk.parity ^ 1], __float_as_uint(m));
        if (f > 0.f) atomicMax(&st->amax_f32_tb, __float_as_uint(f));
        if (e) atomicOr(&st->err, e);
        __threadfence();
        const unsigned done = atomicAdd(&st->blocks_done, 1u);
        if (done == (unsigned)(bk.ctas - 1)) {
            __threadfence();
            finalize_pair(bk, dt);
        }
    }
}

// Where one two-half-step tile reads and writes: the stage of parity
// `parity` in in32 (n_old cells), the intermediate stage (n_mid cells, never
// stored), the final stage in out32 (n_new = n_old cells); the tile's final
// cells start at f0.
struct PairIO {
    const float* in32;
    float* out32;
    long long pitch;
    long long n_old, n_mid, n_new;
    long long f0;
    int parity;
    int bc;
};

// One tile of two staggered half-steps (temporal blocking, FP32 variants):
// stage n (parity p) -> n + 1/2 -> n + 1 (parity p), both with the step lam2.
// The tile owns final cells f0 .. f0 + kTileTB - 1; it loads the parents
// o0 = f0 - 1 .. o0 + 2 kThreadsMixed - 1, builds the intermediate cells
// m0 = o0 + p .. m0 + 2 kThreadsMixed - 2 in registers (each thread's two
// intermediate cells are the parents it needs next, slot for slot), and from
// them the final cells.  Neighbouring tiles build one intermediate cell
// twice.  At a transmissive boundary the intermediate cells outside the stage
// take the adjacent cell's values (the ghost rule of Sec. 2.1's staggered
// mesh), at a periodic one they are the wrapped cells, built from wrapped
// parents.  Returns the largest speeds of the thread's intermediate and final
// cells (cells outside the stages count as 0) and error bits; synchronises
// the block, and the caller synchronises it again before rec is written.
template <int SYS, int P, bool COMP, bool PARK = (P >= 3)>
__device__ __forceinline__ void mixed_pair_tile(const PairIO& io, const ff2 lam2, const StepArgs& args, float2* rec,
                                                float& mid_speed, float& fin_speed, unsigned& err) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    const int t = threadIdx.x;
    const int p = io.parity;
    const long long f0 = io.f0;
    const long long o0 = f0 - 1;
    const long long m0 = o0 + p;

    ff2 ub[NV];
    f2 c[NV][K];
    {
        const TileIO io1{io.in32, nullptr, io.pitch, io.n_old, io.n_mid, m0, p, io.bc};
        mixed_load_parents<SYS, P, COMP>(io1, ub, c);
        mixed_parent_records<SYS, P, COMP, PARK>(ub, c, lam2, args, rec);
    }
    __syncthreads();
    {
        f2 d[NV][K];
        mixed_new_cells<SYS, P, COMP>(rec, args, ub, d, err);
        // intermediate cells m0 + t (lane x) and m0 + t + kThreadsMixed (lane
        // y; slot 2 kThreadsMixed - 1 is not a cell of the tile)
        const long long ia = m0 + t, ib = ia + kThreadsMixed;
        const bool va = ia >= 0 && ia < io.n_mid;
        const bool vb = t < kThreadsMixed - 1 && ib >= 0 && ib < io.n_mid;
        f2 d0[NV];
        sfor<0, NV>([&](auto V) { d0[decltype(V)::value] = d[decltype(V)::value][0]; });
        mid_speed = mixed_cell_speed<SYS>(ub, d0, va, vb, args, err);
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            sfor<1, K>([&](auto Ki) { c[v][decltype(Ki)::value] = d[v][decltype(Ki)::value]; });
        });
        __syncthreads();  // every record of the first half-step has been read
        if (io.bc == BC_TRANSMISSIVE && (m0 < 0 || m0 + 2 * kThreadsMixed - 1 > io.n_mid)) {
            // edge tiles: slots outside [0, n_mid) copy the edge cell
            constexpr int Q = K + 1;  // hi, lo, c_1..c_P per variable
            float* sc = reinterpret_cast<float*>(rec);
            auto save = [&](int slot, int lane) {
                sfor<0, NV>([&](auto V) {
                    constexpr int v = decltype(V)::value;
                    sc[(v * Q + 0) * 2 * kThreadsMixed + slot] = lane ? ub[v].hi.y() : ub[v].hi.x();
                    sc[(v * Q + 1) * 2 * kThreadsMixed + slot] = lane ? ub[v].lo.y() : ub[v].lo.x();
                    sfor<1, K>([&](auto Ki) {
                        constexpr int k = decltype(Ki)::value;
                        sc[(v * Q + 1 + k) * 2 * kThreadsMixed + slot] = lane ? c[v][k].y() : c[v][k].x();
                    });
                });
            };
            save(t, 0);
            save(t + kThreadsMixed, 1);
            __syncthreads();
            auto fetch = [&](long long idx, int lane) {
                const long long cl = idx < 0 ? 0 : (idx >= io.n_mid ? io.n_mid - 1 : idx);
                if (cl == idx) return;
                const int slot = (int)(cl - m0);
                sfor<0, NV>([&](auto V) {
                    constexpr int v = decltype(V)::value;
                    const float hi = sc[(v * Q + 0) * 2 * kThreadsMixed + slot];
                    const float lo = sc[(v * Q + 1) * 2 * kThreadsMixed + slot];
                    if (lane) {
                        ub[v].hi.v.y = hi;
                        ub[v].lo.v.y = lo;
                    } else {
                        ub[v].hi.v.x = hi;
                        ub[v].lo.v.x = lo;
                    }
                    sfor<1, K>([&](auto Ki) {
                        constexpr int k = decltype(Ki)::value;
                        const float x = sc[(v * Q + 1 + k) * 2 * kThreadsMixed + slot];
                        if (lane) c[v][k].v.y = x; else c[v][k].v.x = x;
                    });
                });
            };
            fetch(m0 + t, 0);
            fetch(m0 + t + kThreadsMixed, 1);
            __syncthreads();
        }
    }
    mixed_parent_records<SYS, P, COMP, PARK>(ub, c, lam2, args, rec);
    __syncthreads();
    ff2 ubn[NV];
    f2 d[NV][K];
    mixed_new_cells<SYS, P, COMP>(rec, args, ubn, d, err);
    const TileIO io2{nullptr, io.out32, io.pitch, io.n_mid, io.n_new, f0, p ^ 1, io.bc};
    const bool va = f0 + t < io.n_new;
    const bool vb = t < kThreadsMixed - 2 && f0 + t + kThreadsMixed < io.n_new;
    fin_speed = mixed_store<SYS, P>(io2, ubn, d, va, vb, args, err);
}

// Two staggered half-steps in one pass over HBM (temporal blocking, FP32
// variants) over a whole stage: args.in32 (parity args.parity) ->
// args.out32, one tile (kTileTB final cells) per CTA, both half-steps with
// the dt of the input stage's bound.  The intermediate stage's bound decides
// whether the pair is taken (finalize_pair); a launch that finds ERR_CFL set
// does nothing.
template <int SYS, int P, bool COMP = true>
__global__ void __launch_bounds__(kThreadsMixed, mixed_min_ctas<P>()) halfstep_mixed2_tb2(const StepArgs args) {
    __shared__ float2 rec[mixed2_smem_float2<SYS, P>()];
    if (args.st->err & ERR_CFL) return;  // an earlier pair was refused: the caller steps singly from there
    const StepSize z = step_size(args);
    const ff2 lam2{f2(z.lam_hi), f2(COMP ? z.lam_lo : 0.f)};
    const PairIO io{args.in32, args.out32, args.pitch, args.n_old, args.n_mid, args.n_new,
                    (long long)blockIdx.x * kTileTB, args.parity, args.bc};
    float mid = 0.f, fin = 0.f;
    unsigned err = 0u;
    mixed_pair_tile<SYS, P, COMP>(io, lam2, args, rec, mid, fin, err);
    const PairBook bk{args.st, args.hist, args.hist_cap, (long long)gridDim.x, args.dx, args.cfl, args.tb_nu_max,
                      args.cfl_mode, args.parity, nullptr, nullptr};
    finish_pair(mid, fin, err, z.dt, bk);
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
