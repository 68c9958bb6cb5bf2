// wcc_scheme.cuh -- device building blocks of the fused WCC half-step
// (Shen & Parsani, arXiv 2104.04347, Sec. 2.1-2.2 and Sec. 4).
//
// Internal representation: Taylor coefficients.  A cell polynomial
// u(xi) = sum_k u_kx xi^k / k!  (xi = (x - x_i)/dx, Eq. 1DPolynomial_Space)
// is held as e_k = u_kx / k!, and the space-time Cauchy-Kovalewski table as
// X[a][b] = dx^a dt^b d_x^a d_t^b u / (a! b!).  In this form products of
// series are plain Cauchy products (no binomial weights), the PDE
// u_t = -f_x becomes X[a][b+1] = -lam (a+1)/(b+1) F[a+1][b], and every
// constant of the scheme (flux-integral weights, central-difference weights,
// smoothness-indicator quadratic form) is a compile-time double folded into
// the instruction stream through the static loops below.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wcc_f2.cuh"

namespace wcc {

enum { ADVECTION = 0, BURGERS = 1, EULER = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1 };
enum { PREC_FP64 = 0, PREC_FP32_MIXED = 1, PREC_FP32 = 2 };

// One CTA stages kThreads parent cells and produces kTile = kThreads - 1 new
// cells: new cell t of the tile sits between parents t and t + 1.
constexpr int kThreads = 128;
constexpr int kTile = kThreads - 1;

// ERR_CFL: the second half-step of a two-half-step launch would exceed its
// CFL bound (the pair is not taken; see halfstep_mixed2_tb2).
enum : unsigned { ERR_NONFINITE = 1u, ERR_POSITIVITY = 2u, ERR_CFL = 4u };

// Device-resident time-marching state (one per solver).
struct DevState {
    // amax_bits[s]: largest characteristic speed of the stage with parity s,
    // as the bit pattern of a non-negative double (integer max == double max).
    unsigned long long amax_bits[2];
    // the same bound as FP32 bits, accumulated by the FP32-mixed kernels (an
    // integer max on the bits of non-negative floats); the last CTA of a
    // launch converts it into amax_bits.
    unsigned int amax_f32[2];
    double t;
    long long step;
    unsigned int blocks_done;  // CTAs finished in the running half-step
    unsigned int err;          // ERR_* bits, sticky
    // dt and lam = dt/dx of the next launch, prepared once by the last CTA of
    // the current launch for the CFL number next_cfl (a launch with another
    // CFL number, or the first one after loading data, derives them itself).
    double next_cfl;
    double next_dt;
    double next_lam;
    float next_lam_hi, next_lam_lo;
    // two half-steps per launch: the bound of the pair's final stage (FP32
    // bits, accumulated like amax_f32) and the largest CFL number a pair's
    // second half-step has taken since the state was loaded
    unsigned int amax_f32_tb;
    unsigned int pad_tb_;
    double tb_nu2_max;
};

// Arguments of one half-step launch.  Plane (v, k) of a stage holds the
// Taylor coefficient e_k of variable v for every cell, pitch elements apart.
// FP64: every plane in *64.  FP32-mixed: plane k = 0 in *64 ([v][cell]),
// planes k >= 1 in *32 ([v][k-1][cell]).
struct StepArgs {
    const double* in64;
    const float* in32;
    double* out64;
    float* out32;
    long long pitch;
    long long n_old;
    long long n_new;
    int parity;   // 0: new[i] from old[i], old[i+1]; 1: from old[i-1], old[i]
    int bc;
    int limiter;
    int alpha_is_two;
    double dx;
    int cfl_mode;     // 1: dt from the CFL number (cfl > 0); 0: dt_fixed
    int pad_;
    unsigned long long cfl_bits;  // bit pattern of cfl (integer comparison, no FP64 pipe)
    double cfl;       // > 0: dt = cfl dx / amax of the stage being advanced
    double dt_fixed;  // used when cfl <= 0, with lam_fixed = dt_fixed / dx
    double lam_fixed;
    double adv;       // advection speed
    double gamma;
    double alpha;
    double eps;
    DevState* st;
    double* hist;     // dt of every half-step, indexed by DevState::step
    long long hist_cap;
    // FP32 copies for the FP32-mixed kernels (hi/lo: float-float split)
    float gamma_f, g1_hi, g1_lo, adv_hi, adv_lo, eps_f, alpha_f;
    float lam_fixed_hi, lam_fixed_lo;
    // two half-steps per launch (halfstep_mixed2_tb2): cells of the
    // intermediate stage, and the largest CFL number its second half-step
    // may take with the pair's dt
    long long n_mid;
    double tb_nu_max;
    // FP32 variants: tiles of the single-half-step kernel per CTA (0: the
    // degree's default)
    int tiles_per_cta;
    int pad2_;
};

// dt and lam of this launch (the same values in every thread).
struct StepSize {
    double dt, lam;
    float lam_hi, lam_lo;
};

__device__ __forceinline__ void split_to_floats(double d, float& hi, float& lo) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
}

// CFL step of a solver state: the value the previous launch prepared when it
// was made for the same CFL number, else derived from the stage bound.
__device__ __forceinline__ StepSize cfl_step_size(const DevState* st, unsigned long long cfl_bits, double cfl,
                                                  double dx, int parity) {
    StepSize z;
    if ((unsigned long long)__double_as_longlong(st->next_cfl) == cfl_bits) {
        z.dt = st->next_dt;
        z.lam = st->next_lam;
        z.lam_hi = st->next_lam_hi;
        z.lam_lo = st->next_lam_lo;
    } else {
        const double amax = __longlong_as_double((long long)st->amax_bits[parity]);
        z.dt = cfl * dx / amax;
        z.lam = z.dt / dx;
        split_to_floats(z.lam, z.lam_hi, z.lam_lo);
    }
    return z;
}

__device__ __forceinline__ StepSize step_size(const StepArgs& args) {
    StepSize z;
    if (args.cfl_mode) {
        z = cfl_step_size(args.st, args.cfl_bits, args.cfl, args.dx, args.parity);
    } else {
        z.dt = args.dt_fixed;
        z.lam = args.lam_fixed;
        z.lam_hi = args.lam_fixed_hi;
        z.lam_lo = args.lam_fixed_lo;
    }
    return z;
}

// ------------------------------------------------------------ static loops

template <int I>
struct Int {
    static constexpr int value = I;
};

// Calls f(Int<B>{}), ..., f(Int<E-1>{}); inside f the index is a constant
// expression (decltype(i)::value), so array indices resolve to registers and
// coefficient functions evaluate at compile time.
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(Int<B>{});
        sfor<B + 1, E>(static_cast<F&&>(f));
    }
}

__host__ __device__ constexpr double cfact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}
__host__ __device__ constexpr double cbinom(int n, int k) { return cfact(n) / (cfact(k) * cfact(n - k)); }
__host__ __device__ constexpr double cpow2(int n) {
    double r = 1.0;
    for (int i = 0; i < (n < 0 ? -n : n); ++i) r = (n < 0) ? r * 0.5 : r * 2.0;
    return r;
}
// (-1/2)^n and (1/2)^n
__host__ __device__ constexpr double chalf(int n, bool negative) {
    return (negative && (n & 1)) ? -cpow2(-n) : cpow2(-n);
}
// int_{-1/2}^{1/2} xi^e dxi
__host__ __device__ constexpr double cmoment(int e) { return (e & 1) ? 0.0 : 1.0 / ((e + 1) * cpow2(e)); }
// Quadratic form of the smoothness indicator (Eq. 1DSmoothIndicator) in
// Taylor coefficients: beta = sum_{j,l >= 1} csmooth(j, l) e_j e_l, because
// d^k u/dxi^k = sum_{j >= k} e_j j!/(j-k)! xi^{j-k} and the dx powers cancel.
__host__ __device__ constexpr double csmooth(int j, int l) {
    double s = 0.0;
    const int m = j < l ? j : l;
    for (int k = 1; k <= m; ++k)
        s += cfact(j) / cfact(j - k) * cfact(l) / cfact(l - k) * cmoment(j + l - 2 * k);
    return s;
}

__host__ __device__ constexpr int nvars(int sys) { return sys == EULER ? 3 : 1; }

// Bit pattern of a double on the host.
inline long long __double_as_longlong_host(double d) {
    long long b;
    __builtin_memcpy(&b, &d, sizeof(b));
    return b;
}

// 1/x: correctly rounded division in FP64; the hardware reciprocal with one
// Newton step (correctly rounded) in FP32.
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// NaN / Inf test on the exponent bits (integer pipe only).
__device__ __forceinline__ bool not_finite(double x) {
    return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool not_finite(float x) {
    return (__float_as_int(x) & 0x7f800000) == 0x7f800000;
}

// ------------------------------------------------ Cauchy-Kovalewski (Eq. 1DCauchy_Kovalewski, Sec. 4)

// Parent-cell quantities shared by the two new cells that touch this parent:
//   A[v]    = ubar_R/2 + lam fbar   (contribution when the parent is the left one)
//   B[v]    = ubar_L/2 - lam fbar   (contribution when it is the right one)
//   vtx[v][k] = Taylor coefficient k of the vertex polynomial at t^{n+1/2}
// so that the new cell average is A[left] + B[right] (Eq. SubEq:1DIntegral
// with Eqs. SubEq:1DCellAVGR, SubEq:1DCellAVGL, Cal1DFlux) and the vertex
// values of Eq. SubEq:Cal_1D_Derivatives_4 are k! vtx[k].
template <int SYS, int P, class R>
struct ParentRecord {
    static constexpr int NV = nvars(SYS);
    R A[NV];
    R B[NV];
    R vtx[NV][P + 1];
};

// Space-time Taylor table X[v][a][b] (a + b <= P) of one cell from its
// Taylor coefficients c, and the flux coefficients F0[v][b] at a = 0.
template <int SYS, int P, class R>
__device__ __forceinline__ void ck_table(const R (&c)[nvars(SYS)][P + 1], R lam, const StepArgs& args,
                                         R (&X)[nvars(SYS)][P + 1][P + 1], R (&F0)[nvars(SYS)][P + 1]) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        sfor<0, K>([&](auto A) { X[v][decltype(A)::value][0] = c[v][decltype(A)::value]; });
    });

    constexpr bool f32 = !is_f64<R>;
    if constexpr (SYS == ADVECTION) {
        const R a = f32 ? (R)args.adv_hi : (R)args.adv;
        const R la = lam * a;
        sfor<0, P>([&](auto Bi) {
            constexpr int b = decltype(Bi)::value;
            sfor<0, P - b>([&](auto Ai) {
                constexpr int aa = decltype(Ai)::value;
                constexpr double w = (aa + 1.0) / (b + 1.0);
                X[0][aa][b + 1] = -(la * (R)w) * X[0][aa + 1][b];
            });
        });
        sfor<0, K>([&](auto Bi) {
            constexpr int b = decltype(Bi)::value;
            F0[0][b] = a * X[0][0][b];
        });
    } else if constexpr (SYS == BURGERS) {
        R F[K][K];
        sfor<0, K>([&](auto Bi) {
            constexpr int b = decltype(Bi)::value;
            // F = u^2/2: Cauchy product, symmetric terms paired.
            sfor<0, K - b>([&](auto Ai) {
                constexpr int aa = decltype(Ai)::value;
                R s = (R)0;
                sfor<0, aa + 1>([&](auto Ii) {
                    constexpr int i = decltype(Ii)::value;
                    sfor<0, b + 1>([&](auto Ji) {
                        constexpr int j = decltype(Ji)::value;
                        constexpr int i2 = aa - i, j2 = b - j;
                        // visit each unordered pair once
                        if constexpr (i * (b + 1) + j < i2 * (b + 1) + j2) {
                            s = fma(X[0][i][j], X[0][i2][j2], s);
                        } else if constexpr (i == i2 && j == j2) {
                            s = fma((R)0.5 * X[0][i][j], X[0][i][j], s);
                        }
                    });
                });
                F[aa][b] = s;
            });
            if constexpr (b < P) {
                sfor<0, P - b>([&](auto Ai) {
                    constexpr int aa = decltype(Ai)::value;
                    constexpr double w = (aa + 1.0) / (b + 1.0);
                    X[0][aa][b + 1] = -(lam * (R)w) * F[aa + 1][b];
                });
            }
            F0[0][b] = F[0][b];
        });
    } else {
        // Euler, U = (rho, m, E): velocity w = m / rho by series division,
        // q = m w, p = (gamma - 1)(E - q/2), H = E + p, F = (m, q + p, H w).
        const R g1 = f32 ? (R)args.g1_hi : (R)(args.gamma - 1.0);
        R w[K][K] = {}, H[K][K] = {}, Fm[K][K] = {}, FE[K][K] = {};
        const R inv_rho = recip(X[0][0][0]);
        sfor<0, K>([&](auto Bi) {
            constexpr int b = decltype(Bi)::value;
            sfor<0, K - b>([&](auto Ai) {
                constexpr int aa = decltype(Ai)::value;
                R s = X[1][aa][b];
                sfor<0, aa + 1>([&](auto Ii) {
                    constexpr int i = decltype(Ii)::value;
                    sfor<0, b + 1>([&](auto Ji) {
                        constexpr int j = decltype(Ji)::value;
                        if constexpr (i != 0 || j != 0) s = fma(-X[0][i][j], w[aa - i][b - j], s);
                    });
                });
                w[aa][b] = s * inv_rho;
                R q = (R)0;
                sfor<0, aa + 1>([&](auto Ii) {
                    constexpr int i = decltype(Ii)::value;
                    sfor<0, b + 1>([&](auto Ji) {
                        constexpr int j = decltype(Ji)::value;
                        q = fma(X[1][i][j], w[aa - i][b - j], q);
                    });
                });
                const R p = g1 * fma((R)-0.5, q, X[2][aa][b]);
                H[aa][b] = X[2][aa][b] + p;
                Fm[aa][b] = q + p;
                R fe = (R)0;
                sfor<0, aa + 1>([&](auto Ii) {
                    constexpr int i = decltype(Ii)::value;
                    sfor<0, b + 1>([&](auto Ji) {
                        constexpr int j = decltype(Ji)::value;
                        fe = fma(H[i][j], w[aa - i][b - j], fe);
                    });
                });
                FE[aa][b] = fe;
            });
            if constexpr (b < P) {
                sfor<0, P - b>([&](auto Ai) {
                    constexpr int aa = decltype(Ai)::value;
                    constexpr double wgt = (aa + 1.0) / (b + 1.0);
                    const R lw = lam * (R)wgt;
                    X[0][aa][b + 1] = -lw * X[1][aa + 1][b];
                    X[1][aa][b + 1] = -lw * Fm[aa + 1][b];
                    X[2][aa][b + 1] = -lw * FE[aa + 1][b];
                });
            }
            F0[0][b] = X[1][0][b];
            F0[1][b] = Fm[0][b];
            F0[2][b] = FE[0][b];
        });
    }
}

template <int SYS, int P, class R>
__device__ __forceinline__ void parent_record(const R (&c)[nvars(SYS)][P + 1], R lam, const StepArgs& args,
                                              ParentRecord<SYS, P, R>& out) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    R X[NV][K][K];
    R F0[NV][K];
    ck_table<SYS, P, R>(c, lam, args, X, F0);

    sfor<0, NV>([&](auto V) {
        constexpr int v = decltype(V)::value;
        // Eq. Cal1DFlux in Taylor form: fbar = sum_b F[0][b] / (b + 1).
        R fbar = F0[v][0];
        sfor<1, K>([&](auto Bi) {
            constexpr int b = decltype(Bi)::value;
            fbar = fma((R)(1.0 / (b + 1.0)), F0[v][b], fbar);
        });
        // Eqs. SubEq:1DCellAVGR / SubEq:1DCellAVGL: half-cell averages.
        R ur = c[v][0], ul = c[v][0];
        sfor<1, K>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            constexpr double wk = 1.0 / ((k + 1.0) * cpow2(k));
            ur = fma((R)wk, c[v][k], ur);
            ul = fma((R)((k & 1) ? -wk : wk), c[v][k], ul);
        });
        out.A[v] = fma(lam, fbar, (R)0.5 * ur);
        out.B[v] = fma(-lam, fbar, (R)0.5 * ul);
        // Eq. SubEq:Cal_1D_Derivatives_4: vertex values at t^{n+1/2}.
        sfor<0, K>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;
            R s = X[v][k][0];
            sfor<1, K - k>([&](auto Mi) { s += X[v][k][decltype(Mi)::value]; });
            out.vtx[v][k] = s;
        });
    });
}

// ------------------------------------------------------ new-cell update

// Derivatives from high to low order (Eq. SubEq:Cal_1D_Derivatives_3) and
// the point value (Eq. 1DCalU), in Taylor coefficients:
//   e_{k+1} = (vR_k - vL_k - sum_{m>=3 odd} 2 C(k+m, m) 2^-m e_{k+m}) / (k+1)
//   e_0     = ubar - sum_{k>=2 even} e_k / ((k+1) 2^k)
template <int P, class R>
__device__ __forceinline__ void derivatives_and_point_value(R ubar, const R (&vL)[P + 1], const R (&vR)[P + 1],
                                                            R (&e)[P + 1]) {
    sfor<0, P>([&](auto Ii) {
        constexpr int k = P - 1 - decltype(Ii)::value;
        R s = vR[k] - vL[k];
        sfor<3, P - k + 1>([&](auto Mi) {
            constexpr int m = decltype(Mi)::value;
            if constexpr (m & 1) {
                constexpr double cm = 2.0 * cbinom(k + m, m) * cpow2(-m);
                s = fma((R)-cm, e[k + m], s);
            }
        });
        e[k + 1] = (k == 0) ? s : s * (R)(1.0 / (k + 1.0));
    });
    R u0 = ubar;
    sfor<2, P + 1>([&](auto Ki) {
        constexpr int k = decltype(Ki)::value;
        if constexpr ((k & 1) == 0) u0 = fma((R)(-1.0 / ((k + 1.0) * cpow2(k))), e[k], u0);
    });
    e[0] = u0;
}

// WENO-type limiter of Sec. 2.2 on one scalar (or characteristic) component.
// e: Taylor coefficients of u_0 (overwritten by u_*), ubar its cell average,
// vl / vr the time-extrapolated vertex values u_{i-1/2}, u_{i+1/2}.
template <int P, class R>
__device__ __forceinline__ void limit_scalar(R (&e)[P + 1], R ubar, R vl, R vr, const StepArgs& args) {
    const R s1 = (R)2 * (ubar - vl);   // Eq. SubEq:1DU12, slope of u_1
    const R s2 = (R)2 * (vr - ubar);   // slope of u_2
    // beta_0 (Eq. 1DSmoothIndicator) as a quadratic form in e_1..e_P
    R b0 = (R)0;
    sfor<1, P + 1>([&](auto Ji) {
        constexpr int j = decltype(Ji)::value;
        R row = (R)0;
        sfor<j, P + 1>([&](auto Li) {
            constexpr int l = decltype(Li)::value;
            constexpr double cjl = (l == j ? 1.0 : 2.0) * csmooth(j, l);
            if constexpr (cjl != 0.0) row = fma((R)cjl, e[l], row);
        });
        b0 = fma(row, e[j], b0);
    });
    const R b1 = s1 * s1, b2 = s2 * s2;
    const R eps = (R)args.eps;
    R w0, w1, w2;
    if (args.alpha_is_two) {
        // Multiplied through by the denominators, so that one reciprocal
        // normalises the weights; w0 = 1 - w1 - w2 is exactly 1 when the
        // other two vanish.
        R h0, h1, h2;
        if constexpr (P == 1) {
            // Eq. 1D2ndOrderWeights: w_m ~ (beta_m + eps)^-2
            const R d0 = b0 + eps, d1 = b1 + eps, d2 = b2 + eps;
            const R p12 = d1 * d2, p02 = d0 * d2, p01 = d0 * d1;
            h0 = p12 * p12;
            h1 = p02 * p02;
            h2 = p01 * p01;
        } else {
            // Eq. 1DHighOrderWeights: w0 ~ 1 + (st/d0)^2, w_m ~ (st/d_m)^2
            R up = e[0], um = e[0];
            sfor<1, P + 1>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                up = fma((R)chalf(k, false), e[k], up);
                um = fma((R)chalf(k, true), e[k], um);
            });
            const R rr = up - vr, rl = um - vl;
            const R sigma = fma(rr, rr, rl * rl);
            const R tp = (R)cfact(P) * e[P];
            const R st = sigma * (tp * tp);
            const R d0 = fma(b0, b0, eps), d1 = fma(b1, b1, eps), d2 = fma(b2, b2, eps);
            const R p12 = d1 * d2, p02 = d0 * d2, p01 = d0 * d1;
            const R s12 = st * p12, s02 = st * p02, s01 = st * p01;
            h0 = fma(d0 * p12, d0 * p12, s12 * s12);
            h1 = s02 * s02;
            h2 = s01 * s01;
        }
        const R inv = recip(h0 + h1 + h2);
        w1 = h1 * inv;
        w2 = h2 * inv;
        w0 = (R)1 - (w1 + w2);
    } else {
        R wh0, wh1, wh2;
        if constexpr (P == 1) {
            const R al = (R)args.alpha;
            wh0 = pow((R)1 / (b0 + eps), al); wh1 = pow((R)1 / (b1 + eps), al); wh2 = pow((R)1 / (b2 + eps), al);
        } else {
            R up = e[0], um = e[0];
            sfor<1, P + 1>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                up = fma((R)chalf(k, false), e[k], up);
                um = fma((R)chalf(k, true), e[k], um);
            });
            const R rr = up - vr, rl = um - vl;
            const R sigma = fma(rr, rr, rl * rl);
            const R tp = (R)cfact(P) * e[P];
            const R st = sigma * (tp * tp);
            const R al = (R)args.alpha;
            wh0 = (R)1 + pow(st / fma(b0, b0, eps), al);
            wh1 = pow(st / fma(b1, b1, eps), al);
            wh2 = pow(st / fma(b2, b2, eps), al);
        }
        const R inv = (R)1 / (wh0 + wh1 + wh2);
        w1 = wh1 * inv;
        w2 = wh2 * inv;
        w0 = (R)1 - (w1 + w2);
    }
    // Eq. 1DLimitedPolynomial, coefficient by coefficient.
    e[0] = fma(w0, e[0], (w1 + w2) * ubar);
    e[1] = fma(w0, e[1], fma(w1, s1, w2 * s2));
    sfor<2, P + 1>([&](auto Ki) { e[decltype(Ki)::value] *= w0; });
}

// Eigenvectors of the Euler flux Jacobian at the cell average (conserved
// variables; columns of R for u - c, u, u + c; the textbook closed form cited
// in Sec. 5.2) -- used by the characteristic limiter of Sec. 4.  With
// b1 = (gamma - 1)/c^2, b2 = b1 u^2/2 and H = (E + p)/rho:
//   R = [[1, 1, 1], [u - c, u, u + c], [H - u c, u^2/2, H + u c]],
//   L = [[(b2 + u/c)/2, -(b1 u + 1/c)/2, b1/2],
//        [1 - b2,        b1 u,           -b1 ],
//        [(b2 - u/c)/2, -(b1 u - 1/c)/2, b1/2]].
// Multiplied out, the products need only seven scalars:
//   L d = (X - Y, d_0 - 2 X, X + Y),  X = (b1/2) (u^2/2 d_0 - u d_1 + d_2),
//                                     Y = (1/(2c)) (d_1 - u d_0),
//   R w = (s + w_1, u (s + w_1) + m, H s + u m + u^2/2 w_1),
//         s = w_0 + w_2,  m = c (w_2 - w_0),
// eight multiply-adds per product instead of nine, and a basis of seven
// registers (pairs) instead of fifteen.
template <class R>
struct EulerChar {
    R u, nu, hu2, c, H, b1h, ich;

    __device__ __forceinline__ void left(R d0, R d1, R d2, R (&w)[3]) const {
        const R X = b1h * fma(nu, d1, fma(hu2, d0, d2));
        const R Y = ich * fma(nu, d0, d1);
        w[0] = X - Y;
        w[1] = fma((R)-2, X, d0);
        w[2] = X + Y;
    }
    __device__ __forceinline__ void right(R w0, R w1, R w2, R& d0, R& d1, R& d2) const {
        const R s = w0 + w2;
        const R m = c * (w2 - w0);
        d0 = s + w1;
        d1 = fma(u, d0, m);
        d2 = fma(H, s, fma(u, m, hu2 * w1));
    }
};

// Basis at the conserved state U; false for a non-positive density or
// pressure.
template <class R>
__device__ __forceinline__ bool euler_char(const R (&U)[3], R gamma, EulerChar<R>& E) {
    constexpr bool f32 = !is_f64<R>;
    const R irho = recip(U[0]);
    const R u = U[1] * irho;
    const R g1 = gamma - (R)1;
    const R p = g1 * fma((R)-0.5 * U[1], u, U[2]);
    const R c2 = gamma * p * irho;
    R ic;
    if constexpr (f32) {
        ic = rsqrt_approx(c2);  // the basis only needs FP32 accuracy
        E.c = c2 * ic;
    } else {
        E.c = sqrt(c2);
        ic = (R)1 / E.c;
    }
    E.u = u;
    E.nu = -u;
    E.hu2 = (R)0.5 * u * u;
    E.H = (U[2] + p) * irho;
    E.b1h = (R)0.5 * g1 * ic * ic;
    E.ich = (R)0.5 * ic;
    return all_pos(U[0]) && all_pos(p);
}

// Characteristic speed |u| (Burgers), |a| (advection) or |u| + c (Euler)
// at the centre point values; sets err bits for non-physical states.
template <int SYS, class R>
__device__ __forceinline__ R wave_speed(const R* u0, const StepArgs& args, unsigned& err) {
    constexpr bool f32 = !is_f64<R>;
    if constexpr (SYS == ADVECTION) {
        return f32 ? (R)fabsf(args.adv_hi) : (R)fabs(args.adv);
    } else if constexpr (SYS == BURGERS) {
        return fabs(u0[0]);
    } else {
        const R gamma = f32 ? (R)args.gamma_f : (R)args.gamma;
        const R g1 = f32 ? (R)args.g1_hi : (R)(args.gamma - 1.0);
        const R rho = u0[0];
        if constexpr (f32) {
            const R irho = recip(rho);
            const R u = u0[1] * irho;
            const R p = g1 * fma((R)-0.5 * u0[1], u, u0[2]);
            if (!all_pos(rho) || !all_pos(p)) err |= ERR_POSITIVITY;
            const R c2 = gamma * p * irho;
            return fabs(u) + c2 * rsqrt_approx(c2);
        } else {
            const R irho = (R)1 / rho;
            const R u = u0[1] * irho;
            const R p = g1 * fma((R)-0.5 * u0[1], u, u0[2]);
            if (!all_pos(rho) || !all_pos(p)) err |= ERR_POSITIVITY;
            return fabs(u) + sqrt(gamma * p * irho);
        }
    }
}

}  // namespace wcc
