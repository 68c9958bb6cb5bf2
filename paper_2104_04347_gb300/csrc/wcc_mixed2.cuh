// wcc_mixed2.cuh -- the FP32-mixed half-step with two cells per thread.
//
// Same arithmetic as the scalar FP32-mixed formulation (float-float cell
// averages, leading flux and vertex values; FP32 for the rest; limiter in
// deviation form), but every thread carries a pair of cells in the two lanes
// of the paired FP32 instructions: lane x works on parent t / new cell t of
// the tile, lane y on parent t + kThreads / new cell t + kThreads.  A tile
// has 2 kThreads parents and kTileMixed = 2 kThreads - 1 new cells.  Parent
// records are stored interleaved ((slot t, slot t + kThreads) at index t) so
// that a new cell's two parents are one 64-bit shared-memory load each.
#pragma once

#include "wcc_f2.cuh"
#include "wcc_ff.cuh"
#include "wcc_halfstep_mixed.cuh"

namespace wcc {

constexpr int kTileMixed = 2 * kThreads - 1;

// Resident CTAs per SM the FP32-mixed kernels are compiled for (register
// budget 65536 / (kThreads * kMixedMinCtas) per thread).
#ifndef WCC_MIXED_MIN_CTAS
#define WCC_MIXED_MIN_CTAS 5
#endif
constexpr int kMixedMinCtas = WCC_MIXED_MIN_CTAS;

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

__device__ __forceinline__ ff2 ff2_neg(ff2 a) { return ff2{-a.hi, -a.lo}; }
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return ff2_add(a, ff2_neg(b)); }
__device__ __forceinline__ ff2 ff2_scale(ff2 a, float pow2) { return ff2{a.hi * f2(pow2), a.lo * f2(pow2)}; }

__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
    const f2 p = a.hi * b.hi;
    const f2 e = fma(a.hi, b.hi, -p);
    return fast_two_sum2(p, fma(a.hi, b.lo, fma(a.lo, b.hi, e)));
}

__device__ __forceinline__ ff2 ff2_div(ff2 a, ff2 b) {
    const f2 q1 = fdiv_fast(a.hi, b.hi);
    const f2 p = b.hi * q1;
    const f2 e = fma(b.hi, q1, -p);
    const ff2 bq = fast_two_sum2(p, fma(b.lo, q1, e));
    const ff2 r = ff2_sub(a, bq);
    const f2 q2 = fdiv_fast(r.hi, b.hi);
    return fast_two_sum2(q1, q2);
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
    static __device__ __forceinline__ ff2 add(ff2 a, f2 b) { return ff2_add(a, b); }
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

// Normalised weights in scale-free form (see weights_hi_f32); w0 is formed as
// 1 - w1 - w2 so that it is exactly 1 whenever the other two vanish.
__device__ __forceinline__ void weights_hi_f2(f2 b0, f2 b1, f2 b2, f2 st, const StepArgs& args, f2& w0, f2& w1,
                                              f2& w2) {
    const f2 eps(args.eps_f), tiny(1.4e-45f);
    const f2 d0 = fmax(fma(b0, b0, eps), tiny), d1 = fmax(fma(b1, b1, eps), tiny), d2 = fmax(fma(b2, b2, eps), tiny);
    const f2 dmin = fmin(d0, fmin(d1, d2));
    const f2 q0 = fdiv_fast(dmin, d0), q1 = fdiv_fast(dmin, d1), q2 = fdiv_fast(dmin, d2);
    const f2 z = fmin(fdiv_fast(dmin, st), f2(1e18f));  // st = 0 gives +inf -> 1e18
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
    const f2 inv = fdiv_fast(f2(1.f), h0 + h1 + h2);
    w1 = h1 * inv;
    w2 = h2 * inv;
    w0 = f2(1.f) - (w1 + w2);
}

__device__ __forceinline__ void weights_p1_f2(f2 b0, f2 b1, f2 b2, const StepArgs& args, f2& w0, f2& w1, f2& w2) {
    const f2 eps(args.eps_f), tiny(1.4e-45f);
    const f2 d0 = fmax(b0 + eps, tiny), d1 = fmax(b1 + eps, tiny), d2 = fmax(b2 + eps, tiny);
    const f2 dmin = fmin(d0, fmin(d1, d2));
    const f2 q0 = fdiv_fast(dmin, d0), q1 = fdiv_fast(dmin, d1), q2 = fdiv_fast(dmin, d2);
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
    const f2 inv = fdiv_fast(f2(1.f), h0 + h1 + h2);
    w1 = h1 * inv;
    w2 = h2 * inv;
    w0 = f2(1.f) - (w1 + w2);
}

// Limiter of Sec. 2.2 in deviation form (see limit_deviation_f32), paired.
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
    return nvars(SYS) * (6 + P) * (kThreads + 1);
}

// One tile of the FP32-mixed half-step, two cells per thread: parents
// io.first_new + s - parity for slots s = 0..2 kThreads - 1, new cells
// io.first_new + c for c = 0..kTileMixed - 1.  rec: mixed2_smem_float2 float2
// of shared memory.  Returns the larger of the thread's two cell speeds
// (cells outside the stage count as 0) and error bits; the caller
// synchronises the block before rec is written again.
template <int SYS, int P, bool COMP>
__device__ __forceinline__ void mixed_tile2(const TileIO& io, const ff lam, const StepArgs& args, float2* rec,
                                            float& speed, unsigned& err) {
    using A = FF<COMP>;
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NP = P + 2;
    constexpr int RV = 6 + P;
    constexpr int W = kThreads + 1;  // row width of rec in float2
    const int t = threadIdx.x;
    const long long first_new = io.first_new;
    const ff2 lam2{f2(lam.hi), f2(COMP ? lam.lo : 0.f)};

    // ---- phase 1: parent records of slots t (lane x) and t + kThreads (lane y)
    {
        const long long base = first_new + t - (io.parity ? 1 : 0);
        const long long pa = parent_index(base, io.n_old, io.bc);
        const long long pb = parent_index(base + kThreads, io.n_old, io.bc);
        f2 c[NV][K];
        ff2 ub[NV], u0[NV];
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
            f2 corr(0.f);
            sfor<2, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                if constexpr ((k & 1) == 0) corr = fma(f2((float)(1.0 / ((k + 1.0) * cpow2(k)))), c[v][k], corr);
            });
            u0[v] = A::add(ub[v], -corr);
            c[v][0] = u0[v].hi;
        });
        f2 X[NV][K][K], F0[NV][K];
        ck_table<SYS, P, f2>(c, lam2.hi, args, X, F0);
        ff2 f0[NV];
        flux_ff2<SYS, COMP>(u0, args, f0);
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            f2 fhigh(0.f);
            sfor<1, K>([&](auto Bi) {
                constexpr int b = decltype(Bi)::value;
                fhigh = fma(f2((float)(1.0 / (b + 1.0))), F0[v][b], fhigh);
            });
            const ff2 fbar = A::add(f0[v], fhigh);
            f2 dodd(0.f);
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                if constexpr (k & 1) dodd = fma(f2((float)(1.0 / ((k + 1.0) * cpow2(k)))), c[v][k], dodd);
            });
            const ff2 g = A::add(A::mul(fbar, lam2), f2(0.5f) * dodd);
            const ff2 half_ub = ff2_scale(ub[v], 0.5f);
            const ff2 Ac = A::add(half_ub, g);
            const ff2 Bc = A::sub(half_ub, g);
            f2 vt0(0.f);
            sfor<1, K>([&](auto Mi) { vt0 += X[v][0][decltype(Mi)::value]; });
            const ff2 v0 = A::add(u0[v], vt0);
            float2* r = rec + v * RV * W;
            f2 vals[RV];
            vals[0] = Ac.hi;
            vals[1] = Ac.lo;
            vals[2] = Bc.hi;
            vals[3] = Bc.lo;
            vals[4] = v0.hi;
            vals[5] = v0.lo;
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                f2 s = X[v][k][0];
                sfor<1, K - k>([&](auto Mi) { s += X[v][k][decltype(Mi)::value]; });
                vals[5 + k] = s;
            });
            sfor<0, RV>([&](auto Ri) {
                constexpr int row = decltype(Ri)::value;
                r[row * W + t] = vals[row].v;
                // slot kThreads (lane y of thread 0) is also the right parent of
                // new cell kThreads - 1 (lane x of the last thread); its y lane
                // repeats the value so that the unused lane sees real data
                if (t == 0) r[row * W + kThreads] = make_float2(vals[row].y(), vals[row].y());
            });
        });
    }
    __syncthreads();

    // ---- phase 2: new cells t (lane x) and t + kThreads (lane y)
    const long long ia = first_new + t;
    const long long ib = first_new + kThreads + t;
    const bool va = ia < io.n_new;
    const bool vb = (t < kThreads - 1) && ib < io.n_new;
    ff2 ubn[NV];
    f2 d[NV][K], dl[NV], dr[NV];
    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        const float2* r = rec + v * RV * W;
        const ff2 Ac{f2(r[0 * W + t]), f2(r[1 * W + t])};
        const ff2 Bc{f2(r[2 * W + t + 1]), f2(r[3 * W + t + 1])};
        const ff2 vL0{f2(r[4 * W + t]), f2(r[5 * W + t])};
        const ff2 vR0{f2(r[4 * W + t + 1]), f2(r[5 * W + t + 1])};
        ubn[v] = A::add(Ac, Bc);  // Eq. SubEq:1DIntegral
        dl[v] = A::diff(ubn[v], vL0);
        dr[v] = A::diff(vR0, ubn[v]);
        f2 vL[K], vR[K];
        vL[0] = f2(0.f);
        vR[0] = A::diff(vR0, vL0);
        sfor<1, K>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            vL[k] = f2(r[(5 + k) * W + t]);
            vR[k] = f2(r[(5 + k) * W + t + 1]);
        });
        derivatives_and_point_value<P, f2>(f2(0.f), vL, vR, d[v]);
    });

    if (args.limiter) {
        if constexpr (NV == 1) {
            limit_deviation_f2<P>(d[0], dl[0], dr[0], args);
        } else {
            f2 ubf[3] = {ubn[0].hi, ubn[1].hi, ubn[2].hi};
            EulerEigen<f2> E;
            if (!euler_eigen<f2>(ubf, f2(args.gamma_f), E)) err |= ERR_POSITIVITY;
            f2 cd[3][K], cdl[3], cdr[3];
            sfor<0, 3>([&](auto Ii) {
                constexpr int rr = decltype(Ii)::value;
                cdl[rr] = fma(E.L[rr][0], dl[0], fma(E.L[rr][1], dl[1], E.L[rr][2] * dl[2]));
                cdr[rr] = fma(E.L[rr][0], dr[0], fma(E.L[rr][1], dr[1], E.L[rr][2] * dr[2]));
                sfor<0, K>([&](auto Ki) {
                    constexpr int k = decltype(Ki)::value;
                    cd[rr][k] = fma(E.L[rr][0], d[0][k], fma(E.L[rr][1], d[1][k], E.L[rr][2] * d[2][k]));
                });
                limit_deviation_f2<P>(cd[rr], cdl[rr], cdr[rr], args);
            });
            sfor<0, 3>([&](auto Vi) {
                constexpr int v = decltype(Vi)::value;
                sfor<0, K>([&](auto Ki) {
                    constexpr int k = decltype(Ki)::value;
                    d[v][k] = fma(E.Rm[v][0], cd[0][k], fma(E.Rm[v][1], cd[1][k], E.Rm[v][2] * cd[2][k]));
                });
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
__global__ void __launch_bounds__(kThreads, kMixedMinCtas) halfstep_mixed2(const StepArgs args) {
    __shared__ float2 rec[mixed2_smem_float2<SYS, P>()];
    const StepSize z = step_size(args);
    const TileIO io{args.in32, args.out32, args.pitch, args.n_old, args.n_new,
                    (long long)blockIdx.x * kTileMixed, args.parity, args.bc};
    float speed = 0.f;
    unsigned err = 0u;
    mixed_tile2<SYS, P, COMP>(io, ff_make(z.lam_hi, z.lam_lo), args, rec, speed, err);
    finish_halfstep<float>(speed, err, z.dt, args);
}

}  // namespace wcc
