// wcc2d_scheme.cuh -- device arithmetic of the 2D WCC half-step (Sec. 3.1,
// Sec. 3.2, Sec. 4 and Appendix B of arXiv 2104.04347), in the compute type
// T (double or float).
//
// DOFs are the paper's scaled derivatives u_{kx,ly} = dx^k dy^l d^k_x d^l_y u
// at the cell centre (Eq. 2DPolynomial_Space), k + l <= P, at position
// q = (k+l)(k+l+1)/2 + l of a variable's block.  Space-time series are kept
// as cubes X[k][l][m] (dx^k dy^l dt^m d^k_x d^l_y d^m_t), of which only the
// entries with k + l + m <= P are ever touched; every loop is unrolled so that
// each entry is a register and each coefficient a compile-time constant.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>
#include <utility>

#include "wcc_ff.cuh"

namespace wcc2d {

enum { ADVECTION = 0, BURGERS = 1, EULER = 2 };
enum { PERIODIC = 0, TRANSMISSIVE = 1 };
enum : unsigned { ERR_NONFINITE = 1u, ERR_POSITIVITY = 2u, ERR_BOUNDS = 4u /* checked build only */ };

__host__ __device__ constexpr int nvars(int sys) { return sys == EULER ? 4 : 1; }
__host__ __device__ constexpr int nq(int P) { return (P + 1) * (P + 2) / 2; }
__host__ __device__ constexpr int qidx(int k, int l) { return (k + l) * (k + l + 1) / 2 + l; }
// total degree d and the pair (k, l) stored at position q
__host__ __device__ constexpr int qdeg(int q) {
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= q) ++d;
    return d;
}
__host__ __device__ constexpr int ql_of(int q) { return q - qdeg(q) * (qdeg(q) + 1) / 2; }
__host__ __device__ constexpr int qk_of(int q) { return qdeg(q) - ql_of(q); }
__host__ __device__ constexpr double factd(int n) { return n <= 1 ? 1.0 : n * factd(n - 1); }
__host__ __device__ constexpr double binomd(int n, int k) { return factd(n) / (factd(k) * factd(n - k)); }
__host__ __device__ constexpr double pow2m(int n) { return n <= 0 ? 1.0 : 0.5 * pow2m(n - 1); }  // 2^-n
__host__ __device__ constexpr double sgnd(int k) { return (k & 1) ? -1.0 : 1.0; }              // (-1)^k
__host__ __device__ constexpr double ipow(double x, int n) { return n <= 0 ? 1.0 : x * ipow(x, n - 1); }

// mean of xi^e over [-1/2, 1/2]
__host__ __device__ constexpr double moment(int e) { return (e & 1) ? 0.0 : pow2m(e) / (e + 1); }

// Coefficient of c_q c_q2 in the smoothness indicator of Eq.
// 2DSmoothIndicator (scaled form: the mean over the cell of the squared
// xi/eta-derivatives of every order 1..P), for q = (a, b), q2 = (a2, b2).
__host__ __device__ constexpr double beta_coef(int P, int a, int b, int a2, int b2) {
    double s = 0.0;
    for (int k = 0; k <= P; ++k)
        for (int l = 0; k + l <= P; ++l) {
            if (k + l == 0 || a < k || b < l || a2 < k || b2 < l) continue;
            s += moment(a - k + a2 - k) * moment(b - l + b2 - l) /
                 (factd(a - k) * factd(b - l) * factd(a2 - k) * factd(b2 - l));
        }
    return s;
}

// Value at a vertex (sx/2, sy/2) of the monomial with scaled derivative
// u_{ax,by}: (sx/2)^a (sy/2)^b / (a! b!).
__host__ __device__ constexpr double vertex_coef(int a, int b, int sx, int sy) {
    return ipow(0.5 * sx, a) * ipow(0.5 * sy, b) / (factd(a) * factd(b));
}

// Physical constants and options a kernel needs.
struct Law2D {
    double ax, ay;     // advection velocity
    double gamma;      // Euler
    double alpha, eps; // limiter weights
    int limiter;
};

// 1/x and sqrt(x) for a positive normal x: FP64 as printed (IEEE division
// and square root); FP32 from the hardware estimates, the reciprocal refined
// by one Newton step (within an ulp or two)
template <class T>
__device__ __forceinline__ T recip_t(T x) {
    if constexpr (sizeof(T) == 8) {
        return (T)1 / x;
    } else {
        const float r = __fdividef(1.f, x);
        return fmaf(r, fmaf(-x, r, 1.f), r);
    }
}
template <class T>
__device__ __forceinline__ T sqrt_t(T x) {
    if constexpr (sizeof(T) == 8)
        return sqrt(x);
    else
        return x * rsqrtf(x);
}

template <class T>
__device__ __forceinline__ T weight_pow(T x, T alpha) {
    if constexpr (sizeof(T) == 8)
        return alpha == 2.0 ? x * x : pow(x, alpha);
    else
        return alpha == 2.0f ? x * x : exp2f(alpha * log2f(x));
}

// FP32 ratio a / b of the limiter weights for 0 < a <= b: one approximate
// reciprocal (no division sequence, no branch).  b is kept at or above the
// smallest normal float, which only changes denominators below 1.2e-38,
// where the candidate is flat to rounding.
__device__ __forceinline__ float weight_ratio(float a, float b) { return __fdividef(a, fmaxf(b, 0x1p-126f)); }

// ------------------------------------------------------------------ parent

// What an old cell contributes to the four new cells it touches, per
// variable v:
//   c[v][r]: its share of the cell average of Eq. 2DIntegral in the new cell
//            of which it is vertex r (0: lower left, 1: lower right, 2: upper
//            right, 3: upper left), i.e. a quarter of the quarter average
//            (Eqs. SubEq:2DCellAVGRU ... LD) plus lamx/2 and lamy/2 times its
//            time-averaged edge fluxes (Eqs. SubEq:2DFluxFU ... GL) with the
//            signs of Eq. 2DIntegral;
//   V[v][q]: scaled derivatives at the centre at t^{n+1/2}, k + l <= P - 1
//            (the entries Eqs. SubEq:2DUx, SubEq:2DUy read; q = 0 is the
//            vertex value of the limiter), Eq. SubEq:2DUij.
template <int SYS, int P, class T, bool MX = false>
struct Parent {
    static constexpr int NV = nvars(SYS);
    static constexpr int NQ1 = nq(P - 1);
    T c[NV][4];
    T V[NV][NQ1];
    // FP32-mixed (MX): the parts left in float once the leading terms are
    // taken out to be added in float-float.  The quarter averages of Eqs.
    // SubEq:2DCellAVGRU ... LD are the cell average (their even terms) plus
    // +-odd[v][0] +- odd[v][1] +- odd[v][2], the sums over the terms odd in
    // xi only, in eta only and in both; fl[v][0..3] = the edge fluxes f_U, f_D,
    // g_R, g_L without their leading term f(u_00) (resp. g(u_00)); V[v][0]
    // is without the point value u_00 itself.
    T odd[NV][4];
    T fl[NV][4];
};

// Compile-time loop: f(std::integral_constant<int, I>{}) for I = 0 .. N-1, so
// that every index the body forms is a constant (loops whose bounds depend on
// an outer index are not reliably unrolled by #pragma unroll, and a run-time
// index into a register array sends it to local memory).
template <class F, int... I>
__device__ __forceinline__ void unroll_seq(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void unroll(F&& f) {
    unroll_seq(f, std::make_integer_sequence<int, (N > 0 ? N : 0)>{});
}

// Cauchy-Kovalewski procedure in 2D (Sec. 3.1; Sec. 4 for systems) in
// scaled form, U_{k,l,m+1} = -lamx F_{k+1,l,m} - lamy G_{k,l+1,m}, with the
// Leibniz rule for products and quotients (Dyson / Dumbser-Munz).  Each flux
// entry is used as soon as it is formed: for the next time level of U and
// for the edge-flux integrals of Appendix B.
template <int SYS, int P, class T, bool MX = false>
__device__ __forceinline__ void parent_terms(const T (&q)[nvars(SYS)][nq(P)], T lamx, T lamy, const Law2D& law,
                                             Parent<SYS, P, T, MX>& out) {
    constexpr int NV = nvars(SYS);
    // qa[v]: quarter averages RU, RD, LU, LD at t^n (mean of xi^k over [0, 1/2]
    // is 1/((k+1) 2^k), (-1)^k that over [-1/2, 0]); fl[v]: f_U, f_D on the
    // line x = x_i and g_R, g_L on the line y = y_j, averaged over the half step
    T qa[NV][4], fl[NV][4];
    unroll<NV>([&](auto vc) {
        constexpr int v = vc;
        T ru = 0, rd = 0, lu = 0, ld = 0;
        unroll<P + 1>([&](auto kc) {
            constexpr int k = kc;
            unroll<P + 1 - k>([&](auto lc) {
                constexpr int l = lc;
                const T cd = (T)(pow2m(k) / factd(k + 1) * pow2m(l) / factd(l + 1)) * q[v][qidx(k, l)];
                if constexpr (MX) {
                    // ru, rd, lu collect the terms odd in xi only, in eta only, in both
                    if constexpr ((k & 1) && !(l & 1)) ru += cd;
                    if constexpr (!(k & 1) && (l & 1)) rd += cd;
                    if constexpr ((k & 1) && (l & 1)) lu += cd;
                } else {
                    ru += cd;
                    rd += (T)sgnd(l) * cd;
                    lu += (T)sgnd(k) * cd;
                    ld += (T)(sgnd(k) * sgnd(l)) * cd;
                }
            });
        });
        qa[v][0] = ru;
        qa[v][1] = rd;
        qa[v][2] = lu;
        qa[v][3] = ld;
        fl[v][0] = fl[v][1] = fl[v][2] = fl[v][3] = 0;
    });

    T U[NV][P + 1][P + 1][P + 1];
    T w1[P + 1][P + 1][P + 1], w2[P + 1][P + 1][P + 1], Ep[P + 1][P + 1][P + 1];
    float2 W[P + 1][P + 1][P + 1];  // plain FP32: the velocities (w1, w2) as pairs
    unroll<NV>([&](auto vc) {
        unroll<P + 1>([&](auto kc) {
            unroll<P + 1 - kc>([&](auto lc) { U[vc][kc][lc][0] = q[vc][qidx(kc, lc)]; });
        });
    });

    unroll<P + 1>([&](auto mc) {
        constexpr int m = mc;
        unroll<NV>([&](auto vc) {
            unroll<P - m>([&](auto kc) {
                unroll<P - m - kc>([&](auto lc) { U[vc][kc][lc][m + 1] = 0; });
            });
        });
        unroll<P + 1 - m>([&](auto kc) {
            constexpr int k = kc;
            unroll<P + 1 - m - k>([&](auto lc) {
                constexpr int l = lc;
                T F[NV], G[NV];
                if constexpr (SYS == ADVECTION) {
                    F[0] = (T)law.ax * U[0][k][l][m];
                    G[0] = (T)law.ay * U[0][k][l][m];
                } else if constexpr (SYS == BURGERS) {
                    T s = 0;
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                s += (T)(binomd(k, i) * binomd(l, j) * binomd(m, n)) * U[0][i][j][n] *
                                     U[0][k - i][l - j][m - n];
                            });
                        });
                    });
                    F[0] = (T)0.5 * s;
                    G[0] = F[0];
                } else if constexpr (sizeof(T) == 4 && !MX) {
                    // plain FP32: the two velocities, (q_xx, q_xy) and the two
                    // energy fluxes two at a time in paired FP32 instructions
                    // (FFMA2); the same operations as the scalar form below.
                    // The FP32-mixed kernel keeps the scalar form: there the
                    // pairs cost registers (spills) and it ran slower.
                    float2 s12 = make_float2(U[1][k][l][m], U[2][k][l][m]);
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                if constexpr (i + j + n != 0) {
                                    const float c = (float)(binomd(k, i) * binomd(l, j) * binomd(m, n)) * U[0][i][j][n];
                                    s12 = __ffma2_rn(make_float2(-c, -c), W[k - i][l - j][m - n], s12);
                                }
                            });
                        });
                    });
                    const float inv_rho = recip_t(U[0][0][0][0]);
                    W[k][l][m] = __fmul2_rn(s12, make_float2(inv_rho, inv_rho));
                    float2 qx = make_float2(0.f, 0.f);
                    float qyy = 0.f;
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                const float c = (float)(binomd(k, i) * binomd(l, j) * binomd(m, n));
                                const float a1 = c * U[1][i][j][n], a2 = c * U[2][i][j][n];
                                qx = __ffma2_rn(make_float2(a1, a1), W[k - i][l - j][m - n], qx);
                                qyy = fmaf(a2, W[k - i][l - j][m - n].y, qyy);
                            });
                        });
                    });
                    const float p = (float)(law.gamma - 1.0) * (U[3][k][l][m] - 0.5f * (qx.x + qyy));
                    Ep[k][l][m] = U[3][k][l][m] + p;
                    float2 e12 = make_float2(0.f, 0.f);
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                const float c = (float)(binomd(k, i) * binomd(l, j) * binomd(m, n)) * Ep[i][j][n];
                                e12 = __ffma2_rn(make_float2(c, c), W[k - i][l - j][m - n], e12);
                            });
                        });
                    });
                    F[0] = U[1][k][l][m];
                    F[1] = qx.x + p;
                    F[2] = qx.y;
                    F[3] = e12.x;
                    G[0] = U[2][k][l][m];
                    G[1] = qx.y;
                    G[2] = qyy + p;
                    G[3] = e12.y;
                } else {
                    // velocities from rho w = momentum, solved entry by entry
                    T s1 = U[1][k][l][m], s2 = U[2][k][l][m];
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                if constexpr (i + j + n != 0) {
                                    const T c = (T)(binomd(k, i) * binomd(l, j) * binomd(m, n)) * U[0][i][j][n];
                                    s1 -= c * w1[k - i][l - j][m - n];
                                    s2 -= c * w2[k - i][l - j][m - n];
                                }
                            });
                        });
                    });
                    const T inv_rho = recip_t(U[0][0][0][0]);
                    w1[k][l][m] = s1 * inv_rho;
                    w2[k][l][m] = s2 * inv_rho;
                    T qxx = 0, qxy = 0, qyy = 0;
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                const T c = (T)(binomd(k, i) * binomd(l, j) * binomd(m, n));
                                const T a1 = c * U[1][i][j][n], a2 = c * U[2][i][j][n];
                                qxx += a1 * w1[k - i][l - j][m - n];
                                qxy += a1 * w2[k - i][l - j][m - n];
                                qyy += a2 * w2[k - i][l - j][m - n];
                            });
                        });
                    });
                    const T p = (T)(law.gamma - 1.0) * (U[3][k][l][m] - (T)0.5 * (qxx + qyy));
                    Ep[k][l][m] = U[3][k][l][m] + p;
                    T e1 = 0, e2 = 0;
                    unroll<k + 1>([&](auto i) {
                        unroll<l + 1>([&](auto j) {
                            unroll<m + 1>([&](auto n) {
                                const T c = (T)(binomd(k, i) * binomd(l, j) * binomd(m, n)) * Ep[i][j][n];
                                e1 += c * w1[k - i][l - j][m - n];
                                e2 += c * w2[k - i][l - j][m - n];
                            });
                        });
                    });
                    F[0] = U[1][k][l][m];
                    F[1] = qxx + p;
                    F[2] = qxy;
                    F[3] = e1;
                    G[0] = U[2][k][l][m];
                    G[1] = qxy;
                    G[2] = qyy + p;
                    G[3] = e2;
                }
                unroll<NV>([&](auto vc) {
                    constexpr int v = vc;
                    (void)v;
                    // (k + l >= 1 implies m + 1 <= P)
                    if constexpr (k >= 1) U[v][k - 1][l][m + 1] -= lamx * F[v];
                    if constexpr (l >= 1) U[v][k][l - 1][m + 1] -= lamy * G[v];
                    // Eqs. SubEq:2DFluxFU ... GL: one space direction along the edge, and time
                    if constexpr (k == 0 && (!MX || l + m > 0)) {
                        const T cs = (T)(pow2m(l) / factd(l + 1) / factd(m + 1)) * F[v];
                        fl[v][0] += cs;
                        fl[v][1] += (T)sgnd(l) * cs;
                    }
                    if constexpr (l == 0 && (!MX || k + m > 0)) {
                        const T cs = (T)(pow2m(k) / factd(k + 1) / factd(m + 1)) * G[v];
                        fl[v][2] += cs;
                        fl[v][3] += (T)sgnd(k) * cs;
                    }
                });
            });
        });
    });
    // shares of the new cell averages (Eq. 2DIntegral): as vertex 1 the parent
    // gives RU, +f_U, +g_R; as 2: LU, -f_U, +g_L; as 3: LD, -f_D, -g_L; as 4: RD, +f_D, -g_R
    unroll<NV>([&](auto vc) {
        constexpr int v = vc;
        if constexpr (MX) {
            out.odd[v][0] = qa[v][0];  // odd in xi only
            out.odd[v][1] = qa[v][1];  // odd in eta only
            out.odd[v][2] = qa[v][2];  // odd in both
#pragma unroll
            for (int s = 0; s < 4; ++s) out.fl[v][s] = fl[v][s];
        } else {
            const T hx = (T)0.5 * lamx, hy = (T)0.5 * lamy;
            out.c[v][0] = (T)0.25 * qa[v][0] + hx * fl[v][0] + hy * fl[v][2];
            out.c[v][1] = (T)0.25 * qa[v][2] - hx * fl[v][0] + hy * fl[v][3];
            out.c[v][2] = (T)0.25 * qa[v][3] - hx * fl[v][1] - hy * fl[v][3];
            out.c[v][3] = (T)0.25 * qa[v][1] + hx * fl[v][1] - hy * fl[v][2];
        }
    });
    // Eq. SubEq:2DUij
    unroll<NV>([&](auto vc) {
        unroll<P>([&](auto kc) {
            unroll<P - kc>([&](auto lc) {
                constexpr int k = kc, l = lc;
                T s = 0;
                unroll<P + 1 - k - l>([&](auto mc) {
                    if constexpr (!MX || k + l + mc > 0) s += (T)(1.0 / factd(mc)) * U[vc][k][l][mc];
                });
                out.V[vc][qidx(k, l)] = s;
            });
        });
    });
}

// ---------------------------------------------------------------- new cell

// The linear part of a new cell (Sec. 3.1) from its four parents in the
// vertex order of Eq. 2DTaylorSeries (1 lower left, 2 lower right, 3 upper
// right, 4 upper left): the cell average (Eq. 2DIntegral), the derivatives
// from the highest degree down (Eqs. SubEq:2DUx, SubEq:2DUy, mixed ones as
// the mean of both), the point value (Eq. SubEq:2DCellAVG).  rd.c(r, v) and
// rd.V(r, v, q) read the terms of parent r (struct Parent).
template <int SYS, int P, class T, class Rd>
__device__ __forceinline__ void linear_cell(const Rd& rd, T (&D)[nvars(SYS)][nq(P)], T (&ubar)[nvars(SYS)]) {
    constexpr int NV = nvars(SYS);
    unroll<NV>([&](auto vc) {
        constexpr int v = vc;
        ubar[v] = (rd.c(0, v) + rd.c(1, v)) + (rd.c(2, v) + rd.c(3, v));
        // degree d = P down to 1; within a degree b = d - a runs 0..d
        unroll<P>([&](auto dd) {
            constexpr int d = P - dd;
            unroll<d + 1>([&](auto bc) {
                constexpr int b = bc, a = d - b;
                T sum = 0;
                if constexpr (a >= 1) {  // Eq. SubEq:2DUx with (k, l) = (a - 1, b)
                    constexpr int k = a - 1, l = b, r = P - k - l;
                    constexpr int q0 = qidx(k, l);
                    T s = (T)0.5 * ((rd.V(1, v, q0) + rd.V(2, v, q0)) - (rd.V(0, v, q0) + rd.V(3, v, q0)));
                    unroll<r - 2>([&](auto s3c) {
                        constexpr int s3 = s3c + 3;
                        s -= (T)((pow2m(s3) - ipow(-0.5, s3)) / factd(s3)) * D[v][qidx(k + s3, l)];
                    });
                    unroll<r - 1>([&](auto tc) {
                        constexpr int t = tc + 2;
                        unroll<r - t>([&](auto sc) {
                            constexpr int s1 = sc + 1;
                            if constexpr ((s1 & 1) && !(t & 1))
                                s -= (T)(2.0 * pow2m(s1 + t) / (factd(s1) * factd(t))) * D[v][qidx(k + s1, l + t)];
                        });
                    });
                    sum += s;
                }
                if constexpr (b >= 1) {  // Eq. SubEq:2DUy with (k, l) = (a, b - 1)
                    constexpr int k = a, l = b - 1, r = P - k - l;
                    constexpr int q0 = qidx(k, l);
                    T s = (T)0.5 * ((rd.V(3, v, q0) + rd.V(2, v, q0)) - (rd.V(0, v, q0) + rd.V(1, v, q0)));
                    unroll<r - 2>([&](auto t3c) {
                        constexpr int t3 = t3c + 3;
                        s -= (T)((pow2m(t3) - ipow(-0.5, t3)) / factd(t3)) * D[v][qidx(k, l + t3)];
                    });
                    unroll<r>([&](auto tc) {
                        constexpr int t = tc + 1;
                        unroll<r - t - 1>([&](auto sc) {
                            constexpr int s2 = sc + 2;
                            if constexpr ((t & 1) && !(s2 & 1))
                                s -= (T)(2.0 * pow2m(s2 + t) / (factd(s2) * factd(t))) * D[v][qidx(k + s2, l + t)];
                        });
                    });
                    sum += s;
                }
                D[v][qidx(a, b)] = (a >= 1 && b >= 1) ? (T)0.5 * sum : sum;
            });
        });
        T s = ubar[v];
        unroll<P + 1>([&](auto kc) {
            unroll<P + 1 - kc>([&](auto lc) {
                constexpr int k = kc, l = lc;
                if constexpr (k + l > 0 && !(k & 1) && !(l & 1))
                    s -= (T)(pow2m(k) / factd(k + 1) * pow2m(l) / factd(l + 1)) * D[v][qidx(k, l)];
            });
        });
        D[v][0] = s;
    });
}

// ----------------------------------------------------------------- limiter

// Limiter of Sec. 3.2 for one scalar component: d (the DOFs of u_0, replaced
// by those of u_*), its cell average ub and the vertex values vv[0..3] at
// vertices 1..4.  FP64 follows the printed weights; in FP32 the same weights
// are formed from ratios (every term divided by the largest) so that the
// tiny epsilon cannot overflow them.
template <int P, class T>
__device__ __forceinline__ void limit_scalar(T (&d)[nq(P)], T ub, const T (&vv)[4], const Law2D& law) {
    constexpr int NQ = nq(P);
    T sx[5], sy[5];
    sx[1] = (T)2 * ub - (vv[0] + vv[3]);
    sy[1] = vv[3] - vv[0];
    sx[2] = vv[1] - vv[0];
    sy[2] = (T)2 * ub - (vv[0] + vv[1]);
    sx[3] = (vv[1] + vv[2]) - (T)2 * ub;
    sy[3] = vv[2] - vv[1];
    sx[4] = vv[2] - vv[3];
    sy[4] = (vv[3] + vv[2]) - (T)2 * ub;
    T beta[5];
    {
        // the quadratic form of Eq. 2DSmoothIndicator over pairs q1 <= q2, as
        // sum over q1 of d[q1] times an inner sum over q2 (independent chains)
        T b = 0;
        unroll<NQ>([&](auto q1) {
            T inner = 0;
            unroll<NQ>([&](auto q2) {
                if constexpr (q2 >= q1) {
                    constexpr double c = beta_coef(P, qk_of(q1), ql_of(q1), qk_of(q2), ql_of(q2)) * (q1 == q2 ? 1.0 : 2.0);
                    if constexpr (c != 0.0) inner += (T)c * d[q2];
                }
            });
            b += d[q1] * inner;
        });
        beta[0] = b;
    }
#pragma unroll
    for (int m = 1; m <= 4; ++m) beta[m] = sx[m] * sx[m] + sy[m] * sy[m];
    const T alpha = (T)law.alpha, eps = (T)law.eps;
    T w[5];
    if constexpr (P == 1) {
        // Eq. 2D2ndOrderWeights
        if constexpr (sizeof(T) == 8) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                w[m] = weight_pow<T>((T)1 / (beta[m] + eps), alpha);
                s += w[m];
            }
#pragma unroll
            for (int m = 0; m < 5; ++m) w[m] = w[m] / s;
        } else {
            // every weight divided by that of the smallest denominator
            T bmin = beta[0] + eps;
#pragma unroll
            for (int m = 1; m < 5; ++m) bmin = fminf(bmin, beta[m] + eps);
            T s = 0;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                w[m] = weight_pow<T>(weight_ratio(bmin, beta[m] + eps), alpha);
                s += w[m];
            }
            const T is = recip_t(s);  // s >= 1
#pragma unroll
            for (int m = 0; m < 5; ++m) w[m] *= is;
        }
    } else {
        // Eq. 1DHighOrderWeights in the 2D form of Sec. 3.2: sigma from the
        // four vertex residuals, tau from the degree-P derivatives
        T sigma = 0;
        unroll<4>([&](auto r) {
            constexpr int vsx = (r == 1 || r == 2) ? 1 : -1, vsy = (r >= 2) ? 1 : -1;
            T val = 0;
            unroll<NQ>([&](auto qq) {
                constexpr double c = vertex_coef(qk_of(qq), ql_of(qq), vsx, vsy);
                val += (T)c * d[qq];
            });
            const T res = val - vv[r];
            sigma += res * res;
        });
        T tau = 0;
#pragma unroll
        for (int k = 0; k <= P; ++k) tau += d[qidx(k, P - k)] * d[qidx(k, P - k)];
        const T st = sigma * tau;
        if constexpr (sizeof(T) == 8) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                w[m] = weight_pow<T>(st / (beta[m] * beta[m] + eps), alpha);
                if (m == 0) w[m] += (T)1;
                s += w[m];
            }
#pragma unroll
            for (int m = 0; m < 5; ++m) w[m] = w[m] / s;
        } else {
            // divide every weight by (st / dmin)^alpha, dmin the smallest denominator
            T den[5];
            T dmin = (T)INFINITY;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                den[m] = beta[m] * beta[m] + eps;
                dmin = fminf(dmin, den[m]);
            }
            // the "1 +" of w_0, rescaled.  dmin and st both scaled by 2^64
            // (exact), so that a subnormal st (its dmin can be subnormal too:
            // eps = 1e-40) is a normal number for the reciprocal; st above
            // 2^62 gives lead = 0, its value to rounding
            const T lead = weight_pow<T>((dmin * 0x1p64f) * recip_t(st * 0x1p64f), alpha);
            // lead above 2^30 puts the other weights below 5 2^-30 of the
            // sum: w_0 rounds to 1 (this also keeps the sum, and so the
            // reciprocal below, in range)
            if (!(st > (T)0) || !(lead < 0x1p30f)) {
                w[0] = 1;
                w[1] = w[2] = w[3] = w[4] = 0;
            } else {
                T s = 0;
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    w[m] = weight_pow<T>(weight_ratio(dmin, den[m]), alpha);
                    if (m == 0) w[m] += lead;
                    s += w[m];
                }
                const T is = recip_t(s);  // s >= 1
#pragma unroll
                for (int m = 0; m < 5; ++m) w[m] *= is;
            }
        }
    }
    // Eq. 2DLimitedPolynomial
    T l0 = w[0] * d[0], l1 = w[0] * d[1], l2 = w[0] * d[2];
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
        l0 += w[m] * ub;
        l1 += w[m] * sx[m];
        l2 += w[m] * sy[m];
    }
    d[0] = l0;
    d[1] = l1;
    d[2] = l2;
#pragma unroll
    for (int i = 3; i < NQ; ++i) d[i] = w[0] * d[i];
}

// Rotated characteristic limiting for the 2D Euler equations (Sec. 4):
// direction n from the central-difference gradient of rho e (Eq.
// RotatedNormal), eigenvectors of cos(theta) dF/dU + sin(theta) dG/dU at the
// cell average in closed form, the scalar limiter on each characteristic
// component, and back.  Returns false if the average has non-positive
// density or pressure.  With DEV, D[.][0] and vv hold the point and vertex
// values less the average ub (deviation form): the limiter is unchanged by
// a common shift of the average, the point value and the vertex values, so
// the average's projection is left out and the limited D[.][0] is again a
// deviation from ub (which still sets the eigenvectors).
template <int P, class T, bool DEV = false>
__device__ __forceinline__ bool limit_euler(T (&D)[4][nq(P)], const T (&ub)[4], const T (&vv)[4][4], T lamx,
                                            T lamy, const Law2D& law) {
    constexpr int NQ = nq(P);
    T gx = (T)0.5 * ((vv[3][1] + vv[3][2]) - (vv[3][0] + vv[3][3])) * lamx;
    T gy = (T)0.5 * ((vv[3][3] + vv[3][2]) - (vv[3][0] + vv[3][1])) * lamy;
    const T g2 = gx * gx + gy * gy;
    T nx = 1, ny = 0;
    if (g2 > (T)0) {
        if constexpr (sizeof(T) == 8) {
            const T norm = sqrt(g2);
            nx = gx / norm;
            ny = gy / norm;
        } else {
            const T rn = rsqrtf(g2);
            nx = gx * rn;
            ny = gy * rn;
        }
    }
    const T gm1 = (T)(law.gamma - 1.0);
    const T rho = ub[0];
    T u, v, c, H, b1, ic, q2, p;
    if constexpr (sizeof(T) == 8) {
        u = ub[1] / rho;
        v = ub[2] / rho;
        q2 = u * u + v * v;
        p = gm1 * (ub[3] - (T)0.5 * rho * q2);
        if (!(rho > (T)0) || !(p > (T)0)) return false;
        c = sqrt((T)law.gamma * p / rho);
        H = (ub[3] + p) / rho;
        b1 = gm1 / (c * c);
        ic = (T)1 / c;
    } else {
        const T irho = recip_t(rho);
        u = ub[1] * irho;
        v = ub[2] * irho;
        q2 = u * u + v * v;
        p = gm1 * (ub[3] - (T)0.5 * rho * q2);
        if (!(rho > (T)0) || !(p > (T)0)) return false;
        // c and 1/c within an ulp of each other, so that the left and right
        // eigenvectors stay inverse to float rounding (the projection and the
        // back-projection then cancel where the weights are linear)
        c = sqrt_t((T)law.gamma * p * irho);
        ic = recip_t(c);
        H = (ub[3] + p) * irho;
        b1 = gm1 * ic * ic;
    }
    const T un = u * nx + v * ny, ut = -u * ny + v * nx;
    const T b2 = (T)0.5 * b1 * q2;
    const T R[4][4] = {{1, 1, 0, 1},
                       {u - c * nx, u, -ny, u + c * nx},
                       {v - c * ny, v, nx, v + c * ny},
                       {H - c * un, (T)0.5 * q2, ut, H + c * un}};
    const T L[4][4] = {{(T)0.5 * (b2 + un * ic), (T)-0.5 * (b1 * u + nx * ic), (T)-0.5 * (b1 * v + ny * ic), (T)0.5 * b1},
                       {(T)1 - b2, b1 * u, b1 * v, -b1},
                       {-ut, -ny, nx, 0},
                       {(T)0.5 * (b2 - un * ic), (T)-0.5 * (b1 * u - nx * ic), (T)-0.5 * (b1 * v - ny * ic), (T)0.5 * b1}};
    // With DEV the point value less the average is minus the even correction
    // of the DOFs (k, l) != (0, 0) (the limiter keeps the average), a linear
    // map that the projections commute with: it is formed on each side
    // instead of being projected.
    constexpr int Q0 = DEV ? 1 : 0;
    auto even_corr = [](const T (&d)[NQ]) {
        T s = 0;
        unroll<P + 1>([&](auto kc) {
            unroll<P + 1 - kc>([&](auto lc) {
                constexpr int k = kc, l = lc;
                if constexpr (k + l > 0 && !(k & 1) && !(l & 1))
                    s += (T)(pow2m(k) / factd(k + 1) * pow2m(l) / factd(l + 1)) * d[qidx(k, l)];
            });
        });
        return s;
    };
    T cd[4][NQ], cub[4], cvv[4][4];
    if constexpr (sizeof(T) == 4) {
        // FP32: the projections two DOFs (two vertices) at a time in paired
        // FP32 instructions (FFMA2)
        constexpr int NPR = (NQ - Q0) / 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cub[i] = 0;
            if constexpr (!DEV) {
#pragma unroll
                for (int j = 0; j < 4; ++j) cub[i] += L[i][j] * ub[j];
            }
#pragma unroll
            for (int r = 0; r < 4; r += 2) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc = __ffma2_rn(make_float2(L[i][j], L[i][j]), make_float2(vv[j][r], vv[j][r + 1]), acc);
                cvv[i][r] = acc.x;
                cvv[i][r + 1] = acc.y;
            }
#pragma unroll
            for (int pr = 0; pr < NPR; ++pr) {
                const int qq = Q0 + 2 * pr;
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc = __ffma2_rn(make_float2(L[i][j], L[i][j]), make_float2(D[j][qq], D[j][qq + 1]), acc);
                cd[i][qq] = acc.x;
                cd[i][qq + 1] = acc.y;
            }
            if constexpr ((NQ - Q0) & 1) {
                T sum = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) sum += L[i][j] * D[j][NQ - 1];
                cd[i][NQ - 1] = sum;
            }
            if constexpr (DEV) cd[i][0] = -even_corr(cd[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) limit_scalar<P, T>(cd[i], cub[i], cvv[i], law);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int pr = 0; pr < NPR; ++pr) {
                const int qq = Q0 + 2 * pr;
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    acc = __ffma2_rn(make_float2(R[j][i], R[j][i]), make_float2(cd[i][qq], cd[i][qq + 1]), acc);
                D[j][qq] = acc.x;
                D[j][qq + 1] = acc.y;
            }
            if constexpr ((NQ - Q0) & 1) {
                T sum = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) sum += R[j][i] * cd[i][NQ - 1];
                D[j][NQ - 1] = sum;
            }
            if constexpr (DEV) D[j][0] = -even_corr(D[j]);
        }
        return true;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        cub[i] = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) cvv[i][r] = 0;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) cd[i][qq] = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if constexpr (!DEV) cub[i] += L[i][j] * ub[j];
#pragma unroll
            for (int r = 0; r < 4; ++r) cvv[i][r] += L[i][j] * vv[j][r];
#pragma unroll
            for (int qq = Q0; qq < NQ; ++qq) cd[i][qq] += L[i][j] * D[j][qq];
        }
        if constexpr (DEV) cd[i][0] = -even_corr(cd[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) limit_scalar<P, T>(cd[i], cub[i], cvv[i], law);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int qq = Q0; qq < NQ; ++qq) {
            T s = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) s += R[j][i] * cd[i][qq];
            D[j][qq] = s;
        }
        if constexpr (DEV) D[j][0] = -even_corr(D[j]);
    }
    return true;
}

// s_x/dx + s_y/dy at a cell's centre point values (the 2D CFL rate; the
// half step is dt = nu / max of it).  NaN for non-physical Euler states.
template <int SYS, class T>
__device__ __forceinline__ T cfl_rate(const T* centre, const Law2D& law, T idx, T idy) {
    if constexpr (SYS == ADVECTION) {
        return fabs((T)law.ax) * idx + fabs((T)law.ay) * idy;
    } else if constexpr (SYS == BURGERS) {
        return fabs(centre[0]) * (idx + idy);
    } else {
        const T rho = centre[0];
        if constexpr (sizeof(T) == 8) {
            const T u = centre[1] / rho, v = centre[2] / rho;
            const T p = (T)(law.gamma - 1.0) * (centre[3] - (T)0.5 * rho * (u * u + v * v));
            if (!(rho > (T)0) || !(p > (T)0)) return (T)NAN;
            const T c = sqrt((T)law.gamma * p / rho);
            return (fabs(u) + c) * idx + (fabs(v) + c) * idy;
        } else {
            if (!(rho > (T)0)) return (T)NAN;
            const T irho = recip_t(rho), u = centre[1] * irho, v = centre[2] * irho;
            const T p = (T)(law.gamma - 1.0) * (centre[3] - (T)0.5 * rho * (u * u + v * v));
            if (!(p > (T)0)) return (T)NAN;
            const T c = sqrt_t((T)law.gamma * p * irho);
            return (fabs(u) + c) * idx + (fabs(v) + c) * idy;
        }
    }
}

// ------------------------------------------------------------- FP32-mixed

// Float-float pieces of the FP32-mixed 2D path: the cell average, the leading
// flux terms and the vertex point values carry about 48 bits, everything else
// is float (as in the 1D FP32-mixed path).
using wcc::ff;

// a * b as an unnormalised pair (hi, lo): exact product of a.hi, plus a.lo * b
__device__ __forceinline__ ff ffm_lazy(ff a, float b) {
    const ff p = wcc::two_prod(a.hi, b);
    return ff{p.hi, fmaf(a.lo, b, p.lo)};
}
// a + b + c + s + lo for O(1) floats a, b, c, a small float s and a low part
// lo: every addition of a high part is exact (two_sum), its error joins the
// low part, which is renormalised once at the end.
__device__ __forceinline__ ff ff_sum4(float a, float b, float c, float s, float lo) {
    const ff x = wcc::two_sum(a, b);
    const ff y = wcc::two_sum(x.hi, c);
    const ff z = wcc::two_sum(y.hi, s);
    return wcc::fast_two_sum(z.hi, ((lo + x.lo) + y.lo) + z.lo);
}
// a - b - c - d in float-float, in the same way
__device__ __forceinline__ ff ff_rest3(ff a, ff b, ff c, ff d) {
    const ff x = wcc::two_sum(a.hi, -b.hi);
    const ff y = wcc::two_sum(x.hi, -c.hi);
    const ff z = wcc::two_sum(y.hi, -d.hi);
    return wcc::fast_two_sum(z.hi, ((a.lo - b.lo) - (c.lo + d.lo)) + ((x.lo + y.lo) + z.lo));
}
// a + b + c + d in float-float, in the same way
__device__ __forceinline__ ff ff_sum4(ff a, ff b, ff c, ff d) {
    const ff x = wcc::two_sum(a.hi, b.hi);
    const ff y = wcc::two_sum(x.hi, c.hi);
    const ff z = wcc::two_sum(y.hi, d.hi);
    return wcc::fast_two_sum(z.hi, ((a.lo + b.lo) + (c.lo + d.lo)) + ((x.lo + y.lo) + z.lo));
}
// (a + b) - (c + d) rounded to float
__device__ __forceinline__ float ff_diff2(ff a, ff b, ff c, ff d) {
    const ff x = wcc::two_sum(a.hi, b.hi);
    const ff y = wcc::two_sum(x.hi, -c.hi);
    const ff z = wcc::two_sum(y.hi, -d.hi);
    return z.hi + (((a.lo + b.lo) - (c.lo + d.lo)) + ((x.lo + y.lo) + z.lo));
}
// Float-float operations without the closing renormalisation, for results
// that only feed further float-float arithmetic ((hi, lo) with lo a few ulp
// of hi is as exact a representation; every operation here reads both parts).
__device__ __forceinline__ ff ff_add_u(ff a, ff b) {
    const ff s = wcc::two_sum(a.hi, b.hi);
    return ff{s.hi, s.lo + (a.lo + b.lo)};
}
__device__ __forceinline__ ff ff_add_u(ff a, float b) {
    const ff s = wcc::two_sum(a.hi, b);
    return ff{s.hi, s.lo + a.lo};
}
__device__ __forceinline__ ff ff_mul_u(ff a, ff b) {
    const ff p = wcc::two_prod(a.hi, b.hi);
    return ff{p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo))};
}
__device__ __forceinline__ ff ff_scale(ff a, float pow2) { return ff{a.hi * pow2, a.lo * pow2}; }
// a / b for a normal b: q1 = a.hi / b.hi, then the remainder a - b q1 (its
// leading part a.hi - b.hi q1 is exact, Sterbenz) divided by b.hi; one
// reciprocal estimate serves both quotients
__device__ __forceinline__ ff ffdiv_u(ff a, ff b) {
    const float rb = __fdividef(1.f, b.hi);
    const float q1 = a.hi * rb;
    const float p = b.hi * q1;
    const float e = fmaf(b.hi, q1, -p);
    const float rem = (a.hi - p) + (a.lo - fmaf(b.lo, q1, e));
    return ff{q1, rem * rb};
}

// f(u) and g(u) at a point value u given in float-float (the (0,0,0) entries
// of the flux tables, the leading terms of Eqs. SubEq:2DFluxFU ... GL).
template <int SYS>
__device__ __forceinline__ void lead_flux_ff(const ff (&u)[nvars(SYS)], const Law2D& law, ff (&F)[nvars(SYS)],
                                             ff (&G)[nvars(SYS)]) {
    // every result feeds float-float arithmetic again (the shares take
    // hx f, hy g as exact products): no renormalisation in between; the
    // constants (a_x, a_y, gamma - 1) enter as float-float pairs
    auto pair = [](double c) {
        const float h = (float)c;
        return ff{h, (float)(c - (double)h)};
    };
    if constexpr (SYS == ADVECTION) {
        F[0] = ff_mul_u(u[0], pair(law.ax));
        G[0] = ff_mul_u(u[0], pair(law.ay));
    } else if constexpr (SYS == BURGERS) {
        F[0] = ff_scale(ff_mul_u(u[0], u[0]), 0.5f);
        G[0] = F[0];
    } else {
        const ff vx = ffdiv_u(u[1], u[0]), vy = ffdiv_u(u[2], u[0]);
        const ff mu = ff_mul_u(u[1], vx), mv = ff_mul_u(u[1], vy), nv = ff_mul_u(u[2], vy);
        const ff p = ff_mul_u(ff_add_u(u[3], ff_scale(ff_add_u(mu, nv), -0.5f)), pair(law.gamma - 1.0));
        const ff Ep = ff_add_u(u[3], p);
        F[0] = u[1];
        F[1] = ff_add_u(mu, p);
        F[2] = mv;
        F[3] = ff_mul_u(Ep, vx);
        G[0] = u[2];
        G[1] = mv;
        G[2] = ff_add_u(nv, p);
        G[3] = ff_mul_u(Ep, vy);
    }
}

// Sum over the even (k, l) != (0, 0) of the weights of Eq. SubEq:2DCellAVG
// times u_{kx,ly}: the cell average is u_00 plus this.
template <int P>
__device__ __forceinline__ float even_correction(const float (&d)[nq(P)]) {
    float s = 0.f;
    unroll<P + 1>([&](auto kc) {
        unroll<P + 1 - kc>([&](auto lc) {
            constexpr int k = kc, l = lc;
            if constexpr (k + l > 0 && !(k & 1) && !(l & 1))
                s += (float)(pow2m(k) / factd(k + 1) * pow2m(l) / factd(l + 1)) * d[qidx(k, l)];
        });
    });
    return s;
}

// The new cell's linear part in the FP32-mixed form: the cell average as the
// float-float sum of the four parents' shares, the degree-1 derivatives from
// float-float differences of the vertex point values, the rest as
// linear_cell.  rd.cf(r, v), rd.v00(r, v) (float-float) and rd.V(r, v, q)
// (float, q >= 1) read parent r.  D[v][0] receives the point value (hi).
template <int SYS, int P, class Rd>
__device__ __forceinline__ void linear_cell_mx(const Rd& rd, float (&D)[nvars(SYS)][nq(P)], ff (&ubar)[nvars(SYS)]) {
    constexpr int NV = nvars(SYS);
    unroll<NV>([&](auto vc) {
        constexpr int v = vc;
        ubar[v] = ff_sum4(rd.cf(0, v), rd.cf(1, v), rd.cf(2, v), rd.cf(3, v));
        unroll<P>([&](auto dd) {
            constexpr int d = P - dd;
            unroll<d + 1>([&](auto bc) {
                constexpr int b = bc, a = d - b;
                float sum = 0.f;
                if constexpr (a >= 1) {
                    constexpr int k = a - 1, l = b, r = P - k - l;
                    constexpr int q0 = qidx(k, l);
                    float s;
                    if constexpr (q0 == 0)
                        s = 0.5f * ff_diff2(rd.v00(1, v), rd.v00(2, v), rd.v00(0, v), rd.v00(3, v));
                    else
                        s = 0.5f * ((rd.V(1, v, q0) + rd.V(2, v, q0)) - (rd.V(0, v, q0) + rd.V(3, v, q0)));
                    unroll<r - 2>([&](auto s3c) {
                        constexpr int s3 = s3c + 3;
                        s -= (float)((pow2m(s3) - ipow(-0.5, s3)) / factd(s3)) * D[v][qidx(k + s3, l)];
                    });
                    unroll<r - 1>([&](auto tc) {
                        constexpr int t = tc + 2;
                        unroll<r - t>([&](auto sc) {
                            constexpr int s1 = sc + 1;
                            if constexpr ((s1 & 1) && !(t & 1))
                                s -= (float)(2.0 * pow2m(s1 + t) / (factd(s1) * factd(t))) * D[v][qidx(k + s1, l + t)];
                        });
                    });
                    sum += s;
                }
                if constexpr (b >= 1) {
                    constexpr int k = a, l = b - 1, r = P - k - l;
                    constexpr int q0 = qidx(k, l);
                    float s;
                    if constexpr (q0 == 0)
                        s = 0.5f * ff_diff2(rd.v00(3, v), rd.v00(2, v), rd.v00(0, v), rd.v00(1, v));
                    else
                        s = 0.5f * ((rd.V(3, v, q0) + rd.V(2, v, q0)) - (rd.V(0, v, q0) + rd.V(1, v, q0)));
                    unroll<r - 2>([&](auto t3c) {
                        constexpr int t3 = t3c + 3;
                        s -= (float)((pow2m(t3) - ipow(-0.5, t3)) / factd(t3)) * D[v][qidx(k, l + t3)];
                    });
                    unroll<r>([&](auto tc) {
                        constexpr int t = tc + 1;
                        unroll<r - t - 1>([&](auto sc) {
                            constexpr int s2 = sc + 2;
                            if constexpr ((t & 1) && !(s2 & 1))
                                s -= (float)(2.0 * pow2m(s2 + t) / (factd(s2) * factd(t))) * D[v][qidx(k + s2, l + t)];
                        });
                    });
                    sum += s;
                }
                D[v][qidx(a, b)] = (a >= 1 && b >= 1) ? 0.5f * sum : sum;
            });
        });
        D[v][0] = wcc::ff_add(ubar[v], -even_correction<P>(D[v])).hi;
    });
}

}  // namespace wcc2d
