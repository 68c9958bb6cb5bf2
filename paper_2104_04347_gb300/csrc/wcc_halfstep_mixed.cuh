// wcc_halfstep_mixed.cuh -- the FP32-mixed instantiation of the fused
// half-step (no FP64 instruction in the per-cell work).
//
// Storage per variable: the cell average ubar as a float-float pair (two FP32
// planes, hi and lo) and the Taylor coefficients e_1..e_P as FP32 planes
// (e_k = dx^k u^(k) / k!, the scaled form keeps them in range).  Arithmetic:
//   * float-float (compensated FP32) where the result is a small difference
//     of O(1) quantities or must conserve: the leading flux term f(u_0), the
//     flux-integral / half-average contributions A, B of each parent, the new
//     cell average A[left] + B[right] (Eq. SubEq:1DIntegral), and the vertex
//     values u_{i -/+ 1/2} that enter ubar - u_{i-1/2}, u_{i+1/2} - ubar
//     (Eqs. SubEq:1DU12, 1DHighOrderWeights) and e_1;
//   * FP32 for everything else: the Cauchy-Kovalewski table, higher flux and
//     vertex terms, derivatives, the limiter.
// Because the limited polynomial keeps the cell average (Eq.
// 1DLimitedPolynomial), the limiter here works on deviations from ubar only
// and never rounds ubar; sums of ubar telescope exactly up to float-float
// rounding.  The limiter weights are evaluated in a scale-free form (ratios
// to the smallest denominator), so the tiny epsilon of the paper neither
// overflows nor underflows FP32.
#pragma once

#include "wcc_ff.cuh"
#include "wcc_halfstep.cuh"

namespace wcc {

// Normalised weights for P = 1 (Eq. 1D2ndOrderWeights):
// w_m proportional to (1 / (beta_m + eps))^alpha, evaluated as
// ((beta_min + eps) / (beta_m + eps))^alpha <= 1.
__device__ __forceinline__ void weights_p1_f32(float b0, float b1, float b2, const StepArgs& args, float& w0,
                                               float& w1, float& w2) {
    const float eps = args.eps_f;
    const float d0 = b0 + eps, d1 = b1 + eps, d2 = b2 + eps;
    const float dmin = fminf(d0, fminf(d1, d2));
    float q0, q1, q2;
    if (dmin > 0.f) {
        q0 = __fdividef(dmin, d0);
        q1 = __fdividef(dmin, d1);
        q2 = __fdividef(dmin, d2);
    } else {  // eps = 0 and a flat candidate: it takes all the weight
        q0 = (d0 == 0.f) ? 1.f : 0.f;
        q1 = (d1 == 0.f) ? 1.f : 0.f;
        q2 = (d2 == 0.f) ? 1.f : 0.f;
    }
    float h0, h1, h2;
    if (args.alpha_is_two) {
        h0 = q0 * q0; h1 = q1 * q1; h2 = q2 * q2;
    } else {
        const float al = args.alpha_f;
        h0 = __powf(q0, al); h1 = __powf(q1, al); h2 = __powf(q2, al);
    }
    const float inv = __fdividef(1.f, h0 + h1 + h2);
    w0 = h0 * inv; w1 = h1 * inv; w2 = h2 * inv;
}

// Normalised weights for P >= 2 (Eq. 1DHighOrderWeights):
// w0 ~ 1 + (st/d0)^alpha, w_m ~ (st/d_m)^alpha with d = beta^2 + eps,
// multiplied through by (d_min/st)^alpha.
__device__ __forceinline__ void weights_hi_f32(float b0, float b1, float b2, float st, const StepArgs& args,
                                               float& w0, float& w1, float& w2) {
    const float eps = args.eps_f;
    const float d0 = fmaf(b0, b0, eps), d1 = fmaf(b1, b1, eps), d2 = fmaf(b2, b2, eps);
    const float dmin = fminf(d0, fminf(d1, d2));
    if (!(st > 0.f)) {  // sigma tau underflows: the weights of u_1, u_2 vanish
        w0 = 1.f; w1 = 0.f; w2 = 0.f;
        return;
    }
    float q0, q1, q2, z;
    if (dmin > 0.f) {
        q0 = __fdividef(dmin, d0);
        q1 = __fdividef(dmin, d1);
        q2 = __fdividef(dmin, d2);
        z = fminf(__fdividef(dmin, st), 1e18f);
    } else {
        q0 = (d0 == 0.f) ? 1.f : 0.f;
        q1 = (d1 == 0.f) ? 1.f : 0.f;
        q2 = (d2 == 0.f) ? 1.f : 0.f;
        z = 0.f;
    }
    float h0, h1, h2;
    if (args.alpha_is_two) {
        h0 = fmaf(z, z, q0 * q0); h1 = q1 * q1; h2 = q2 * q2;
    } else {
        const float al = args.alpha_f;
        h0 = __powf(z, al) + __powf(q0, al); h1 = __powf(q1, al); h2 = __powf(q2, al);
    }
    const float inv = __fdividef(1.f, h0 + h1 + h2);
    w0 = h0 * inv; w1 = h1 * inv; w2 = h2 * inv;
}

// Limiter of Sec. 2.2 in deviation form.  d[0] = u_0(centre) - ubar,
// d[1..P] = Taylor coefficients; dl = ubar - u_{i-1/2}, dr = u_{i+1/2} - ubar.
// On return d holds the same quantities of the limited polynomial.
template <int P>
__device__ __forceinline__ void limit_deviation_f32(float (&d)[P + 1], float dl, float dr, const StepArgs& args) {
    const float s1 = 2.f * dl, s2 = 2.f * dr;
    float b0 = 0.f;
    sfor<1, P + 1>([&](auto Ji) {
        constexpr int j = decltype(Ji)::value;
        float row = 0.f;
        sfor<j, P + 1>([&](auto Li) {
            constexpr int l = decltype(Li)::value;
            constexpr double cjl = (l == j ? 1.0 : 2.0) * csmooth(j, l);
            if constexpr (cjl != 0.0) row = fmaf((float)cjl, d[l], row);
        });
        b0 = fmaf(row, d[j], b0);
    });
    const float b1 = s1 * s1, b2 = s2 * s2;
    float w0, w1, w2;
    if constexpr (P == 1) {
        weights_p1_f32(b0, b1, b2, args, w0, w1, w2);
    } else {
        float up = d[0], um = d[0];
        sfor<1, P + 1>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            up = fmaf((float)chalf(k, false), d[k], up);
            um = fmaf((float)chalf(k, true), d[k], um);
        });
        const float rr = up - dr;   // u_0(x_{i+1/2}) - u_{i+1/2}
        const float rl = um + dl;   // u_0(x_{i-1/2}) - u_{i-1/2}
        const float sigma = fmaf(rr, rr, rl * rl);
        const float tp = (float)cfact(P) * d[P];
        weights_hi_f32(b0, b1, b2, sigma * (tp * tp), args, w0, w1, w2);
    }
    d[0] *= w0;
    d[1] = fmaf(w0, d[1], fmaf(w1, s1, w2 * s2));
    sfor<2, P + 1>([&](auto Ki) { d[decltype(Ki)::value] *= w0; });
}

// Leading flux term f(u_0) in float-float.
template <int SYS>
__device__ __forceinline__ void flux_ff(const ff (&u)[nvars(SYS)], const StepArgs& args, ff (&f)[nvars(SYS)]) {
    if constexpr (SYS == ADVECTION) {
        f[0] = ff_mul(u[0], ff_make(args.adv_hi, args.adv_lo));
    } else if constexpr (SYS == BURGERS) {
        f[0] = ff_scale(ff_mul(u[0], u[0]), 0.5f);
    } else {
        const ff w = ff_div(u[1], u[0]);
        const ff q = ff_mul(u[1], w);
        const ff p = ff_mul(ff_add(u[2], ff_scale(q, -0.5f)), ff_make(args.g1_hi, args.g1_lo));
        f[0] = u[1];
        f[1] = ff_add(q, p);
        f[2] = ff_mul(ff_add(u[2], p), w);
    }
}

// Shared-memory floats one tile of mixed_tile<SYS, P> needs.
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

template <int SYS, int P>
constexpr int mixed_tile_smem_floats() {
    return nvars(SYS) * (6 + P) * kThreads;
}

// One tile of the FP32-mixed half-step: parents io.first_new + t - parity
// (t = 0..kThreads-1) of the stage io.in32, new cells io.first_new + t
// (t < kTile) of io.out32.  rec: mixed_tile_smem_floats<SYS, P>() floats of
// shared memory.  Returns each thread's characteristic speed (0 for threads
// without a new cell) and error bits.  The caller synchronises the block
// before rec is written again.
template <int SYS, int P>
__device__ __forceinline__ void mixed_tile(const TileIO& io, const ff lam, const StepArgs& args, float* rec,
                                           float& speed, unsigned& err) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NP = P + 2;       // planes per variable: ubar hi, ubar lo, e_1..e_P
    constexpr int RV = 6 + P;       // record per variable: A(2), B(2), v0(2), vtx_1..vtx_P
    const int t = threadIdx.x;
    const long long first_new = io.first_new;

    // ---- phase 1: parent record of parent slot t
    {
        const long long p = parent_index(first_new + t - (io.parity ? 1 : 0), io.n_old, io.bc);
        float c[NV][K];
        ff ub[NV], u0[NV];
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            ub[v].hi = __ldg(io.in32 + (long long)(v * NP + 0) * io.pitch + p);
            ub[v].lo = __ldg(io.in32 + (long long)(v * NP + 1) * io.pitch + p);
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                c[v][k] = __ldg(io.in32 + (long long)(v * NP + k + 1) * io.pitch + p);
            });
            // point value u_0 = ubar - sum_{k even >= 2} e_k / ((k+1) 2^k)  (Eq. 1DCalU)
            float corr = 0.f;
            sfor<2, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                if constexpr ((k & 1) == 0) corr = fmaf((float)(1.0 / ((k + 1.0) * cpow2(k))), c[v][k], corr);
            });
            u0[v] = ff_add(ub[v], -corr);
            c[v][0] = u0[v].hi;
        });
        float X[NV][K][K], F0[NV][K];
        ck_table<SYS, P, float>(c, lam.hi, args, X, F0);
        ff f0[NV];
        flux_ff<SYS>(u0, args, f0);
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            // Eq. Cal1DFlux: fbar = f(u_0) + sum_{b >= 1} F[0][b] / (b + 1)
            float fhigh = 0.f;
            sfor<1, K>([&](auto Bi) {
                constexpr int b = decltype(Bi)::value;
                fhigh = fmaf((float)(1.0 / (b + 1.0)), F0[v][b], fhigh);
            });
            const ff fbar = ff_add(f0[v], fhigh);
            // half-cell averages ubar_R/L = ubar +/- D_odd with
            // D_odd = sum_{k odd} e_k / ((k+1) 2^k)  (Eqs. SubEq:1DCellAVGR/L)
            float dodd = 0.f;
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                if constexpr (k & 1) dodd = fmaf((float)(1.0 / ((k + 1.0) * cpow2(k))), c[v][k], dodd);
            });
            const ff g = ff_add(ff_mul(fbar, lam), 0.5f * dodd);
            const ff half_ub = ff_scale(ub[v], 0.5f);
            const ff A = ff_add(half_ub, g);
            const ff B = ff_sub(half_ub, g);
            // vertex values at t^{n+1/2} (Eq. SubEq:Cal_1D_Derivatives_4)
            float vt0 = 0.f;
            sfor<1, K>([&](auto Mi) { vt0 += X[v][0][decltype(Mi)::value]; });
            const ff v0 = ff_add(u0[v], vt0);
            float* r = rec + v * RV * kThreads;
            r[0 * kThreads + t] = A.hi;
            r[1 * kThreads + t] = A.lo;
            r[2 * kThreads + t] = B.hi;
            r[3 * kThreads + t] = B.lo;
            r[4 * kThreads + t] = v0.hi;
            r[5 * kThreads + t] = v0.lo;
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                float s = X[v][k][0];
                sfor<1, K - k>([&](auto Mi) { s += X[v][k][decltype(Mi)::value]; });
                r[(5 + k) * kThreads + t] = s;
            });
        });
    }
    __syncthreads();

    // ---- phase 2: new cell t from parent slots t (left) and t + 1 (right)
    const long long i = first_new + t;
    speed = 0.f;
    if (t < kTile && i < io.n_new) {
        ff ubn[NV];
        float d[NV][K], dl[NV], dr[NV];
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            const float* r = rec + v * RV * kThreads;
            const ff A = ff_make(r[0 * kThreads + t], r[1 * kThreads + t]);
            const ff B = ff_make(r[2 * kThreads + t + 1], r[3 * kThreads + t + 1]);
            const ff vL0 = ff_make(r[4 * kThreads + t], r[5 * kThreads + t]);
            const ff vR0 = ff_make(r[4 * kThreads + t + 1], r[5 * kThreads + t + 1]);
            ubn[v] = ff_add(A, B);                          // Eq. SubEq:1DIntegral
            dl[v] = ff_diff(ubn[v], vL0);
            dr[v] = ff_diff(vR0, ubn[v]);
            float vL[K], vR[K];
            vL[0] = 0.f;
            vR[0] = ff_diff(vR0, vL0);
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                vL[k] = r[(5 + k) * kThreads + t];
                vR[k] = r[(5 + k) * kThreads + t + 1];
            });
            // derivatives high -> low (Eq. SubEq:Cal_1D_Derivatives_3); with
            // a zero mean d[0] comes out as u_0(centre) - ubar (Eq. 1DCalU)
            derivatives_and_point_value<P, float>(0.f, vL, vR, d[v]);
        });

        if (args.limiter) {
            if constexpr (NV == 1) {
                limit_deviation_f32<P>(d[0], dl[0], dr[0], args);
            } else {
                float ubf[3] = {ubn[0].hi, ubn[1].hi, ubn[2].hi};
                EulerEigen<float> E;
                if (!euler_eigen<float>(ubf, args.gamma_f, E)) err |= ERR_POSITIVITY;
                float cd[3][K], cdl[3], cdr[3];
                sfor<0, 3>([&](auto Ii) {
                    constexpr int r = decltype(Ii)::value;
                    cdl[r] = fmaf(E.L[r][0], dl[0], fmaf(E.L[r][1], dl[1], E.L[r][2] * dl[2]));
                    cdr[r] = fmaf(E.L[r][0], dr[0], fmaf(E.L[r][1], dr[1], E.L[r][2] * dr[2]));
                    sfor<0, K>([&](auto Ki) {
                        constexpr int k = decltype(Ki)::value;
                        cd[r][k] = fmaf(E.L[r][0], d[0][k], fmaf(E.L[r][1], d[1][k], E.L[r][2] * d[2][k]));
                    });
                    limit_deviation_f32<P>(cd[r], cdl[r], cdr[r], args);
                });
                sfor<0, 3>([&](auto Vi) {
                    constexpr int v = decltype(Vi)::value;
                    sfor<0, K>([&](auto Ki) {
                        constexpr int k = decltype(Ki)::value;
                        d[v][k] = fmaf(E.Rm[v][0], cd[0][k], fmaf(E.Rm[v][1], cd[1][k], E.Rm[v][2] * cd[2][k]));
                    });
                });
            }
        }

        float u0[NV];
        float check = 0.f;   // NaN / Inf in any stored value reaches this sum
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            check += ubn[v].hi;
            __stcs(io.out32 + (long long)(v * NP + 0) * io.pitch + i, ubn[v].hi);
            __stcs(io.out32 + (long long)(v * NP + 1) * io.pitch + i, ubn[v].lo);
            sfor<1, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                check += d[v][k];
                __stcs(io.out32 + (long long)(v * NP + k + 1) * io.pitch + i, d[v][k]);
            });
            u0[v] = ubn[v].hi + d[v][0];
        });
        if (not_finite(check)) err |= ERR_NONFINITE;
        speed = wave_speed<SYS, float>(u0, args, err);
    }
}

template <int SYS, int P>
__global__ void __launch_bounds__(kThreads) halfstep_mixed(const StepArgs args) {
    __shared__ float rec[mixed_tile_smem_floats<SYS, P>()];
    const StepSize z = step_size(args);
    const TileIO io{args.in32, args.out32, args.pitch, args.n_old, args.n_new,
                    (long long)blockIdx.x * kTile, args.parity, args.bc};
    float speed = 0.f;
    unsigned err = 0u;
    mixed_tile<SYS, P>(io, ff_make(z.lam_hi, z.lam_lo), args, rec, speed, err);
    finish_halfstep<float>(speed, err, z.dt, args);
}


// Largest characteristic speed of a stored FP32-mixed stage.
template <int SYS, int P>
__global__ void __launch_bounds__(256) stage_speed_mixed(const float* planes, long long pitch, long long n,
                                                          StepArgs args, int slot) {
    constexpr int NV = nvars(SYS);
    constexpr int NP = P + 2;
    double m = 0.0;
    unsigned err = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float u0[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            float corr = 0.f;
#pragma unroll
            for (int k = 2; k <= P; k += 2)
                corr += planes[(long long)(v * NP + k + 1) * pitch + i] / (float)((k + 1) * (1 << k));
            u0[v] = (planes[(long long)(v * NP) * pitch + i] + planes[(long long)(v * NP + 1) * pitch + i]) - corr;
        }
        double s = (double)wave_speed<SYS, float>(u0, args, err);
        if (s != s) {
            s = __longlong_as_double(0x7ff0000000000000ll);
            err |= ERR_NONFINITE;
        }
        m = fmax(m, s);
    }
    m = warp_max<double>(m);
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(&args.st->amax_bits[slot], (unsigned long long)__double_as_longlong(m));
    if (err) atomicOr(&args.st->err, err);
}

}  // namespace wcc
