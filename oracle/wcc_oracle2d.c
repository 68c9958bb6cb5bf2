/*
 * wcc_oracle2d.c -- plain, slow FP64 CPU oracle for the 2D weighted compact
 * central (WCC) half-step of arXiv 2104.04347: the linear scheme of Sec. 3.1
 * (Eqs. 2DIntegral, 2DTaylorSeries, 2DDerivatives, Appendix B), the limiter
 * of Sec. 3.2 (Eqs. 2DLimitedPolynomial ... 1DHighOrderWeights in 2D form)
 * and, for the Euler equations, the rotated characteristic decomposition of
 * Sec. 4 (Eq. RotatedNormal).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  The
 * product path (the CUDA library) shares no code, header, table or helper
 * with it.
 *
 * Conventions (Sec. 3.1):
 *   - DOFs are the scaled derivatives u_{kx,ly} = dx^k dy^l d^k_x d^l_y u at
 *     the cell centre (Eq. 2DPolynomial_Space), k + l <= P, stored
 *     [j][i][var][q] (row j along y, column i along x) with
 *     q = d (d + 1) / 2 + l, d = k + l (by total degree, then by l).
 *   - dt is the HALF step t^{n+1/2} - t^n; lamx = dt/dx, lamy = dt/dy.
 *   - Parity 0 advances an integer stage to the half stage: new (i, j) is
 *     the staggered cell [x_i, x_{i+1}] x [y_j, y_{j+1}] built from old
 *     (i, j), (i+1, j), (i, j+1), (i+1, j+1).  Parity 1 advances a half stage
 *     to the integer stage: new (i, j) is built from old (i-1, j-1), (i, j-1),
 *     (i-1, j), (i, j).
 *   - Periodic: both stages hold nx x ny cells.  Transmissive: the integer
 *     stage holds (nx+1) x (ny+1) cells centred on the grid points, the half
 *     stage nx x ny; a ghost parent is a copy of the nearest cell along each
 *     axis (zeroth-order extrapolation, as in 1D).
 *
 * Written for readability: Leibniz sums in the paper's derivative form,
 * binomials recomputed where used, no blocking or fusion.  Each old cell's
 * Cauchy-Kovalewski expansion and the terms of Eq. 2DIntegral that depend on
 * that cell alone are evaluated once per half-step and then read by its four
 * children.  Compiled with -O2 -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O2_MAXP 4
#define O2_MAXV 4
#define O2_NK (O2_MAXP + 1)
#define O2_MAXQ ((O2_MAXP + 1) * (O2_MAXP + 2) / 2)

enum { O2_ADVECTION = 0, O2_BURGERS = 1, O2_EULER = 2 };
enum { O2_PERIODIC = 0, O2_TRANSMISSIVE = 1 };

/* The conservation law and scheme options.  Field order is part of the
 * ctypes interface in oracle/__init__.py. */
typedef struct {
    int system;    /* O2_ADVECTION (f = ax u, g = ay u), O2_BURGERS (f = g = u^2/2), O2_EULER */
    int P;         /* polynomial degree, 1..4 */
    int limiter;   /* 1: WENO-type limiter of Sec. 3.2 on every new cell */
    int bc;        /* O2_PERIODIC or O2_TRANSMISSIVE */
    double ax, ay; /* advection velocity */
    double gamma;  /* ratio of specific heats (Euler) */
    double alpha;  /* weight exponent */
    double eps;    /* epsilon in the weights, 1e-40 in the paper */
} o2_law;

static int o2_nv(const o2_law* L) { return L->system == O2_EULER ? 4 : 1; }
static int o2_nq(int P) { return (P + 1) * (P + 2) / 2; }
static int o2_idx(int k, int l) { return (k + l) * (k + l + 1) / 2 + l; }

static double o2_fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

static double o2_binom(int n, int k) { return o2_fact(n) / (o2_fact(k) * o2_fact(n - k)); }

static double o2_sgn(int k) { return (k % 2) ? -1.0 : 1.0; } /* (-1)^k */

/* Scaled space-time derivatives X[k][l][m] = dx^k dy^l dt^m d^k_x d^l_y d^m_t X
 * at the cell centre, time level t^n, for k + l + m <= P. */
typedef double o2_series[O2_NK][O2_NK][O2_NK];

/* Generalised Leibniz rule for Z = X Y, entry (a, b, c):
 * Z_abc = sum C(a,i) C(b,j) C(c,n) X_ijn Y_{a-i,b-j,c-n}.  The scalings by
 * dx, dy and dt distribute over the two factors (Sec. 4, Dyson /
 * Dumbser-Munz). */
static double o2_leibniz(o2_series X, o2_series Y, int a, int b, int c) {
    double s = 0.0;
    for (int i = 0; i <= a; ++i)
        for (int j = 0; j <= b; ++j)
            for (int n = 0; n <= c; ++n)
                s += o2_binom(a, i) * o2_binom(b, j) * o2_binom(c, n) * X[i][j][n] * Y[a - i][b - j][c - n];
    return s;
}

/* The quotient W = X / D from X = D W (Leibniz), solved entry by entry in an
 * order where every lower entry is known: W_abc = (X_abc - sum over
 * (i,j,n) != 0 of C C C D_ijn W_{a-i,b-j,c-n}) / D_000. */
static void o2_quotient_entry(o2_series X, o2_series D, o2_series W, int a, int b, int c) {
    double s = X[a][b][c];
    for (int i = 0; i <= a; ++i)
        for (int j = 0; j <= b; ++j)
            for (int n = 0; n <= c; ++n) {
                if (i == 0 && j == 0 && n == 0) continue;
                s -= o2_binom(a, i) * o2_binom(b, j) * o2_binom(c, n) * D[i][j][n] * W[a - i][b - j][c - n];
            }
    W[a][b][c] = s / D[0][0][0];
}

/* Cauchy-Kovalewski procedure in 2D (Sec. 3.1: time derivatives from the
 * PDE u_t = -f_x - g_y, used repeatedly; Sec. 4 for systems).  In scaled
 * form: U_{k,l,m+1} = -lamx F_{k+1,l,m} - lamy G_{k,l+1,m}.  Level m = 0
 * holds the stored DOFs; at each level the flux derivatives follow from the
 * Leibniz rule, then give the next level of U. */
static void o2_cauchy_kovalewski(const o2_law* L, const double* q, double lamx, double lamy,
                                 o2_series U[O2_MAXV], o2_series F[O2_MAXV], o2_series G[O2_MAXV]) {
    const int P = L->P, nv = o2_nv(L), nq = o2_nq(P);
    static const o2_series zero; /* all zeros */
    o2_series w1, w2, qxx, qxy, qyy, p, Ep; /* Euler: velocities, momentum fluxes, pressure, E + p */
    memcpy(w1, zero, sizeof(zero));
    memcpy(w2, zero, sizeof(zero));
    memcpy(qxx, zero, sizeof(zero));
    memcpy(qxy, zero, sizeof(zero));
    memcpy(qyy, zero, sizeof(zero));
    memcpy(p, zero, sizeof(zero));
    memcpy(Ep, zero, sizeof(zero));
    for (int v = 0; v < nv; ++v) {
        memcpy(U[v], zero, sizeof(zero));
        memcpy(F[v], zero, sizeof(zero));
        memcpy(G[v], zero, sizeof(zero));
        for (int k = 0; k <= P; ++k)
            for (int l = 0; k + l <= P; ++l) U[v][k][l][0] = q[v * nq + o2_idx(k, l)];
    }
    for (int m = 0; m <= P; ++m) {
        for (int k = 0; k <= P - m; ++k)
            for (int l = 0; k + l <= P - m; ++l) {
                if (L->system == O2_ADVECTION) {
                    F[0][k][l][m] = L->ax * U[0][k][l][m];
                    G[0][k][l][m] = L->ay * U[0][k][l][m];
                } else if (L->system == O2_BURGERS) {
                    F[0][k][l][m] = 0.5 * o2_leibniz(U[0], U[0], k, l, m);
                    G[0][k][l][m] = F[0][k][l][m];
                } else {
                    /* U = (rho, rho u, rho v, E) */
                    o2_quotient_entry(U[1], U[0], w1, k, l, m);
                    o2_quotient_entry(U[2], U[0], w2, k, l, m);
                    qxx[k][l][m] = o2_leibniz(U[1], w1, k, l, m);
                    qxy[k][l][m] = o2_leibniz(U[1], w2, k, l, m);
                    qyy[k][l][m] = o2_leibniz(U[2], w2, k, l, m);
                    p[k][l][m] = (L->gamma - 1.0) * (U[3][k][l][m] - 0.5 * (qxx[k][l][m] + qyy[k][l][m]));
                    Ep[k][l][m] = U[3][k][l][m] + p[k][l][m];
                    F[0][k][l][m] = U[1][k][l][m];
                    F[1][k][l][m] = qxx[k][l][m] + p[k][l][m];
                    F[2][k][l][m] = qxy[k][l][m];
                    F[3][k][l][m] = o2_leibniz(Ep, w1, k, l, m);
                    G[0][k][l][m] = U[2][k][l][m];
                    G[1][k][l][m] = qxy[k][l][m];
                    G[2][k][l][m] = qyy[k][l][m] + p[k][l][m];
                    G[3][k][l][m] = o2_leibniz(Ep, w2, k, l, m);
                }
            }
        if (m < P)
            for (int k = 0; k <= P - m - 1; ++k)
                for (int l = 0; k + l <= P - m - 1; ++l)
                    for (int v = 0; v < nv; ++v)
                        U[v][k][l][m + 1] = -lamx * F[v][k + 1][l][m] - lamy * G[v][k][l + 1][m];
    }
}

/* What an old cell contributes to the new cells around it (Appendix B and
 * Eq. SubEq:2DUij), per variable:
 *   qa[0..3]: quarter averages at t^n over RU, RD, LU, LD (Eqs. SubEq:2DCellAVGRU ... LD);
 *   fl[0..3]: time-averaged edge fluxes f_U, f_D (on the line x = x_i) and
 *             g_R, g_L (on the line y = y_j) (Eqs. SubEq:2DFluxFU ... GL);
 *   V[q]:     the scaled derivatives at the cell centre at t^{n+1/2}
 *             (Eq. SubEq:2DUij), all k + l <= P. */
typedef struct {
    double qa[O2_MAXV][4];
    double fl[O2_MAXV][4];
    double V[O2_MAXV][O2_MAXQ];
} o2_parent;

enum { O2_RU = 0, O2_RD = 1, O2_LU = 2, O2_LD = 3 };
enum { O2_FU = 0, O2_FD = 1, O2_GR = 2, O2_GL = 3 };

static void o2_parent_terms(const o2_law* L, const double* q, double lamx, double lamy, o2_parent* out) {
    const int P = L->P, nv = o2_nv(L), nq = o2_nq(P);
    o2_series U[O2_MAXV], F[O2_MAXV], G[O2_MAXV];
    o2_cauchy_kovalewski(L, q, lamx, lamy, U, F, G);
    for (int v = 0; v < nv; ++v) {
        for (int s = 0; s < 4; ++s) {
            out->qa[v][s] = 0.0;
            out->fl[v][s] = 0.0;
        }
        for (int k = 0; k <= P; ++k)
            for (int l = 0; k + l <= P; ++l) {
                /* quarter [0, 1/2] or [-1/2, 0] in each direction: the mean of
                 * xi^k over it is (+-1)^k / ((k+1) 2^k) */
                double cx = 1.0 / (o2_fact(k + 1) * ldexp(1.0, k));
                double cy = 1.0 / (o2_fact(l + 1) * ldexp(1.0, l));
                double d = q[v * nq + o2_idx(k, l)];
                out->qa[v][O2_RU] += cx * cy * d;
                out->qa[v][O2_RD] += cx * o2_sgn(l) * cy * d;
                out->qa[v][O2_LU] += o2_sgn(k) * cx * cy * d;
                out->qa[v][O2_LD] += o2_sgn(k) * cx * o2_sgn(l) * cy * d;
            }
        /* flux integrals: one space direction along the edge, time */
        for (int a = 0; a <= P; ++a)
            for (int m = 0; a + m <= P; ++m) {
                double cs = 1.0 / (o2_fact(a + 1) * ldexp(1.0, a));
                double ct = 1.0 / o2_fact(m + 1);
                out->fl[v][O2_FU] += cs * ct * F[v][0][a][m];
                out->fl[v][O2_FD] += o2_sgn(a) * cs * ct * F[v][0][a][m];
                out->fl[v][O2_GR] += cs * ct * G[v][a][0][m];
                out->fl[v][O2_GL] += o2_sgn(a) * cs * ct * G[v][a][0][m];
            }
        for (int k = 0; k <= P; ++k)
            for (int l = 0; k + l <= P; ++l) {
                double s = 0.0;
                for (int m = 0; m <= P - k - l; ++m) s += U[v][k][l][m] / o2_fact(m);
                out->V[v][o2_idx(k, l)] = s;
            }
    }
}

/* Smoothness indicator of a 2D polynomial of degree n with scaled
 * derivatives c[q] (Eq. 2DSmoothIndicator).  With xi = (x - x_i)/dx,
 * eta = (y - y_j)/dy the factors dx^(2k-1) dy^(2l-1) cancel, leaving
 * beta = sum over 1 <= k + l <= n of the integral over [-1/2, 1/2]^2 of
 * (d^k_xi d^l_eta u)^2, where d^k_xi d^l_eta u = sum over a >= k, b >= l of
 * c_ab xi^(a-k) eta^(b-l) / ((a-k)! (b-l)!).  The square is expanded term by
 * term with the moments int xi^e dxi = 1/((e+1) 2^e) for even e, 0 for odd. */
static double o2_moment(int e) { return (e % 2) ? 0.0 : 1.0 / ((double)(e + 1) * ldexp(1.0, e)); }

static double o2_smoothness(const double* c, int n) {
    double beta = 0.0;
    for (int k = 0; k <= n; ++k)
        for (int l = 0; k + l <= n; ++l) {
            if (k + l == 0) continue;
            for (int a = k; a <= n; ++a)
                for (int b = l; a + b <= n; ++b)
                    for (int a2 = k; a2 <= n; ++a2)
                        for (int b2 = l; a2 + b2 <= n; ++b2) {
                            double mx = o2_moment((a - k) + (a2 - k));
                            double my = o2_moment((b - l) + (b2 - l));
                            if (mx == 0.0 || my == 0.0) continue;
                            beta += c[o2_idx(a, b)] * c[o2_idx(a2, b2)] * mx * my /
                                    (o2_fact(a - k) * o2_fact(b - l) * o2_fact(a2 - k) * o2_fact(b2 - l));
                        }
        }
    return beta;
}

/* Value of the polynomial of Eq. 2DPolynomial_Space at (xi, eta). */
static double o2_poly_value(const double* c, int n, double xi, double eta) {
    double s = 0.0;
    for (int k = 0; k <= n; ++k)
        for (int l = 0; k + l <= n; ++l)
            s += c[o2_idx(k, l)] * pow(xi, (double)k) * pow(eta, (double)l) / (o2_fact(k) * o2_fact(l));
    return s;
}

/* Vertices of a new cell in the paper's numbering of Eq. 2DTaylorSeries:
 * 1 = (i, j) lower left, 2 = (i+1, j) lower right, 3 = (i+1, j+1) upper
 * right, 4 = (i, j+1) upper left. */
enum { O2_V1 = 0, O2_V2 = 1, O2_V3 = 2, O2_V4 = 3 };

/* Limiter for one scalar component (Sec. 3.2).
 * d[q]: DOFs of u_0 (Eq. 2DHighOrderPolynomial), overwritten with those of
 * u_*; ubar: cell average of u_0; vv[4]: the vertex values (Eq. SubEq:2DUij)
 * at vertices 1..4.  wout (may be NULL) receives w_0 .. w_4. */
static void o2_limit_scalar(const o2_law* L, double* d, double ubar, const double* vv, double* wout) {
    const int P = L->P, nq = o2_nq(P);
    /* Eq. 2DLowOrderPolynomial: four linear candidates with mean ubar and
     * slopes from the edges left (1), bottom (2), right (3), top (4). */
    double sl[5][2];
    sl[1][0] = 2.0 * ubar - (vv[O2_V1] + vv[O2_V4]);
    sl[1][1] = vv[O2_V4] - vv[O2_V1];
    sl[2][0] = vv[O2_V2] - vv[O2_V1];
    sl[2][1] = 2.0 * ubar - (vv[O2_V1] + vv[O2_V2]);
    sl[3][0] = (vv[O2_V2] + vv[O2_V3]) - 2.0 * ubar;
    sl[3][1] = vv[O2_V3] - vv[O2_V2];
    sl[4][0] = vv[O2_V3] - vv[O2_V4];
    sl[4][1] = (vv[O2_V4] + vv[O2_V3]) - 2.0 * ubar;
    double beta[5];
    beta[0] = o2_smoothness(d, P);
    for (int m = 1; m <= 4; ++m) {
        double c[3] = {ubar, sl[m][0], sl[m][1]}; /* q order: (0,0), (1,0), (0,1) */
        beta[m] = o2_smoothness(c, 1);
    }
    double wh[5];
    if (P == 1) {
        /* Eq. 2D2ndOrderWeights */
        for (int m = 0; m < 5; ++m) wh[m] = pow(1.0 / (beta[m] + L->eps), L->alpha);
    } else {
        /* 2D form of Eq. 1DHighOrderWeights: sigma = residuals at the four
         * vertices between the space polynomial and the time-extrapolated
         * values; tau = sum of the squared degree-P derivatives. */
        const double cx[4] = {-0.5, 0.5, 0.5, -0.5}, cy[4] = {-0.5, -0.5, 0.5, 0.5};
        double sigma = 0.0;
        for (int r = 0; r < 4; ++r) {
            double res = o2_poly_value(d, P, cx[r], cy[r]) - vv[r];
            sigma += res * res;
        }
        double tau = 0.0;
        for (int k = 0; k <= P; ++k) tau += d[o2_idx(k, P - k)] * d[o2_idx(k, P - k)];
        for (int m = 0; m < 5; ++m) wh[m] = pow(sigma * tau / (beta[m] * beta[m] + L->eps), L->alpha);
        wh[0] += 1.0;
    }
    double sum = wh[0] + wh[1] + wh[2] + wh[3] + wh[4];
    double w[5];
    for (int m = 0; m < 5; ++m) w[m] = wh[m] / sum;
    /* Eq. 2DLimitedPolynomial, DOF by DOF */
    double lim[O2_MAXQ];
    lim[0] = w[0] * d[0];
    lim[1] = w[0] * d[1];
    lim[2] = w[0] * d[2];
    for (int m = 1; m <= 4; ++m) {
        lim[0] += w[m] * ubar;
        lim[1] += w[m] * sl[m][0];
        lim[2] += w[m] * sl[m][1];
    }
    for (int i = 3; i < nq; ++i) lim[i] = w[0] * d[i];
    for (int i = 0; i < nq; ++i) d[i] = lim[i];
    if (wout)
        for (int m = 0; m < 5; ++m) wout[m] = w[m];
}

/* Solve R X = I for the 4x4 inverse by Gauss-Jordan elimination with partial
 * pivoting (plain textbook method). */
static void o2_invert4(double R[4][4], double Linv[4][4]) {
    double A[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            A[i][j] = R[i][j];
            A[i][4 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 8; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        double inv = 1.0 / A[c][c];
        for (int j = 0; j < 8; ++j) A[c][j] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            double f = A[r][c];
            for (int j = 0; j < 8; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Linv[i][j] = A[i][4 + j];
}

/* Right eigenvectors of A(U, theta) = cos(theta) dF/dU + sin(theta) dG/dU
 * for the 2D Euler equations in conserved variables (Sec. 4; Toro's
 * textbook form), columns for u_n - c, u_n (entropy), u_n (shear), u_n + c
 * with u_n = u nx + v ny; the left eigenvectors as the matrix inverse.
 * Exposed for tests. */
void oracle2d_euler_eigenvectors(double gamma, const double* U, double nx, double ny, double* Rout,
                                 double* Lout) {
    double rho = U[0], u = U[1] / U[0], v = U[2] / U[0], E = U[3];
    double p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    double c = sqrt(gamma * p / rho);
    double H = (E + p) / rho;
    double un = u * nx + v * ny, ut = -u * ny + v * nx;
    double R[4][4] = {{1.0, 1.0, 0.0, 1.0},
                      {u - c * nx, u, -ny, u + c * nx},
                      {v - c * ny, v, nx, v + c * ny},
                      {H - c * un, 0.5 * (u * u + v * v), ut, H + c * un}};
    double Li[4][4];
    o2_invert4(R, Li);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            Rout[4 * i + j] = R[i][j];
            Lout[4 * i + j] = Li[i][j];
        }
}

/* One new staggered cell from the terms of its four parents, given in the
 * vertex order 1..4 of Eq. 2DTaylorSeries.  Writes the new DOFs [var][q] to
 * out.  Optional diagnostics: weights[nv][5], ubar_out[nv], normal_out[2]
 * (the rotated direction for Euler). */
static void o2_new_cell_from(const o2_law* L, const o2_parent* pv[4], double lamx, double lamy, double* out,
                             double* weights, double* ubar_out, double* normal_out) {
    const int P = L->P, nv = o2_nv(L), nq = o2_nq(P);
    double D[O2_MAXV][O2_MAXQ], ubar[O2_MAXV], vv[O2_MAXV][4];
    const o2_parent *p1 = pv[O2_V1], *p2 = pv[O2_V2], *p3 = pv[O2_V3], *p4 = pv[O2_V4];
    for (int v = 0; v < nv; ++v) {
        /* Eq. 2DIntegral: quarter averages plus fluxes through the four edges */
        ubar[v] = 0.25 * (p1->qa[v][O2_RU] + p4->qa[v][O2_RD] + p2->qa[v][O2_LU] + p3->qa[v][O2_LD]) +
                  0.5 * lamx * (p1->fl[v][O2_FU] + p4->fl[v][O2_FD] - p2->fl[v][O2_FU] - p3->fl[v][O2_FD]) +
                  0.5 * lamy * (p1->fl[v][O2_GR] + p2->fl[v][O2_GL] - p4->fl[v][O2_GR] - p3->fl[v][O2_GL]);
        for (int r = 0; r < 4; ++r) vv[v][r] = pv[r]->V[v][0];
        for (int i = 0; i < nq; ++i) D[v][i] = 0.0;
        /* Eqs. SubEq:2DUx, SubEq:2DUy from the highest degree down; a mixed
         * derivative given by both is their mean (remark after Eq. 2DDerivatives) */
        for (int d = P; d >= 1; --d)
            for (int b = 0; b <= d; ++b) {
                int a = d - b;
                double sum = 0.0;
                int count = 0;
                if (a >= 1) { /* Eq. SubEq:2DUx with (k, l) = (a-1, b) */
                    int k = a - 1, l = b, r = P - k - l;
                    double s = 0.5 * ((p2->V[v][o2_idx(k, l)] + p3->V[v][o2_idx(k, l)]) -
                                      (p1->V[v][o2_idx(k, l)] + p4->V[v][o2_idx(k, l)]));
                    for (int s3 = 3; s3 <= r; ++s3)
                        s -= (ldexp(1.0, -s3) - pow(-0.5, (double)s3)) / o2_fact(s3) * D[v][o2_idx(k + s3, l)];
                    for (int t = 2; t <= r; ++t)
                        for (int s1 = 1; s1 <= r - t; ++s1)
                            s -= 0.5 * (1.0 - o2_sgn(s1)) * (1.0 + o2_sgn(t)) / (o2_fact(s1) * o2_fact(t) * ldexp(1.0, s1 + t)) *
                                 D[v][o2_idx(k + s1, l + t)];
                    sum += s;
                    ++count;
                }
                if (b >= 1) { /* Eq. SubEq:2DUy with (k, l) = (a, b-1) */
                    int k = a, l = b - 1, r = P - k - l;
                    double s = 0.5 * ((p4->V[v][o2_idx(k, l)] + p3->V[v][o2_idx(k, l)]) -
                                      (p1->V[v][o2_idx(k, l)] + p2->V[v][o2_idx(k, l)]));
                    for (int t3 = 3; t3 <= r; ++t3)
                        s -= (ldexp(1.0, -t3) - pow(-0.5, (double)t3)) / o2_fact(t3) * D[v][o2_idx(k, l + t3)];
                    for (int t = 1; t <= r; ++t)
                        for (int s2 = 2; s2 <= r - t; ++s2)
                            s -= 0.5 * (1.0 + o2_sgn(s2)) * (1.0 - o2_sgn(t)) / (o2_fact(s2) * o2_fact(t) * ldexp(1.0, s2 + t)) *
                                 D[v][o2_idx(k + s2, l + t)];
                    sum += s;
                    ++count;
                }
                D[v][o2_idx(a, b)] = sum / (double)count;
            }
        /* Eq. SubEq:2DCellAVG solved for the point value */
        double s = ubar[v];
        for (int k = 0; k <= P; ++k)
            for (int l = 0; k + l <= P; ++l) {
                if (k + l == 0) continue;
                double ck = (1.0 + o2_sgn(k)) / (o2_fact(k + 1) * ldexp(1.0, k + 1));
                double cl = (1.0 + o2_sgn(l)) / (o2_fact(l + 1) * ldexp(1.0, l + 1));
                s -= ck * cl * D[v][o2_idx(k, l)];
            }
        D[v][0] = s;
    }
    if (ubar_out)
        for (int v = 0; v < nv; ++v) ubar_out[v] = ubar[v];

    if (L->limiter) {
        if (nv == 1) {
            o2_limit_scalar(L, D[0], ubar[0], vv[0], weights);
        } else {
            /* Eq. RotatedNormal with phi = rho e (Sec. 5.3): the gradient by
             * central differences of the vertex values of E (the leading
             * terms of Eqs. SubEq:2DUx, SubEq:2DUy), in physical units up to
             * the common factor dt: (dE/dx, dE/dy) dt = (sx lamx, sy lamy).
             * A zero gradient (or dt = 0) takes the x direction. */
            double gx = 0.5 * ((vv[3][O2_V2] + vv[3][O2_V3]) - (vv[3][O2_V1] + vv[3][O2_V4])) * lamx;
            double gy = 0.5 * ((vv[3][O2_V4] + vv[3][O2_V3]) - (vv[3][O2_V1] + vv[3][O2_V2])) * lamy;
            double norm = sqrt(gx * gx + gy * gy);
            double nx = 1.0, ny = 0.0;
            if (norm > 0.0) {
                nx = gx / norm;
                ny = gy / norm;
            }
            if (normal_out) {
                normal_out[0] = nx;
                normal_out[1] = ny;
            }
            double R[16], Lm[16];
            oracle2d_euler_eigenvectors(L->gamma, ubar, nx, ny, R, Lm);
            double cD[O2_MAXV][O2_MAXQ], cub[O2_MAXV], cvv[O2_MAXV][4];
            for (int i = 0; i < 4; ++i) {
                cub[i] = 0.0;
                for (int r = 0; r < 4; ++r) cvv[i][r] = 0.0;
                for (int q = 0; q < nq; ++q) cD[i][q] = 0.0;
                for (int j = 0; j < 4; ++j) {
                    cub[i] += Lm[4 * i + j] * ubar[j];
                    for (int r = 0; r < 4; ++r) cvv[i][r] += Lm[4 * i + j] * vv[j][r];
                    for (int q = 0; q < nq; ++q) cD[i][q] += Lm[4 * i + j] * D[j][q];
                }
            }
            for (int i = 0; i < 4; ++i)
                o2_limit_scalar(L, cD[i], cub[i], cvv[i], weights ? weights + 5 * i : NULL);
            for (int j = 0; j < 4; ++j)
                for (int q = 0; q < nq; ++q) {
                    double s = 0.0;
                    for (int i = 0; i < 4; ++i) s += R[4 * j + i] * cD[i][q];
                    D[j][q] = s;
                }
        }
    }
    for (int v = 0; v < nv; ++v)
        for (int q = 0; q < nq; ++q) out[v * nq + q] = D[v][q];
}

/* One new cell from its four parents' DOFs (vertex order 1..4), for tests. */
void oracle2d_new_cell(const o2_law* L, const double* q1, const double* q2, const double* q3, const double* q4,
                       double lamx, double lamy, double* out, double* weights, double* ubar_out, double* normal_out) {
    o2_parent par[4];
    const double* qs[4] = {q1, q2, q3, q4};
    const o2_parent* pv[4];
    for (int r = 0; r < 4; ++r) {
        o2_parent_terms(L, qs[r], lamx, lamy, &par[r]);
        pv[r] = &par[r];
    }
    o2_new_cell_from(L, pv, lamx, lamy, out, weights, ubar_out, normal_out);
}

/* An old cell's terms, for tests: qa[nv][4], fl[nv][4], V[nv][nq]. */
void oracle2d_parent_terms(const o2_law* L, const double* q, double lamx, double lamy, double* qa, double* fl,
                           double* V) {
    const int nv = o2_nv(L), nq = o2_nq(L->P);
    o2_parent t;
    o2_parent_terms(L, q, lamx, lamy, &t);
    for (int v = 0; v < nv; ++v) {
        for (int s = 0; s < 4; ++s) {
            qa[v * 4 + s] = t.qa[v][s];
            fl[v * 4 + s] = t.fl[v][s];
        }
        for (int i = 0; i < nq; ++i) V[v * nq + i] = t.V[v][i];
    }
}

/* Scaled Cauchy-Kovalewski tables of one cell, for tests: U, F, G as
 * [nv][P+1][P+1][P+1], entry (k, l, m) = dx^k dy^l dt^m d^k_x d^l_y d^m_t. */
void oracle2d_ck_table(const o2_law* L, const double* q, double lamx, double lamy, double* Uo, double* Fo,
                       double* Go) {
    const int nv = o2_nv(L), nk = L->P + 1;
    o2_series U[O2_MAXV], F[O2_MAXV], G[O2_MAXV];
    o2_cauchy_kovalewski(L, q, lamx, lamy, U, F, G);
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < nk; ++k)
            for (int l = 0; l < nk; ++l)
                for (int m = 0; m < nk; ++m) {
                    long o = ((v * nk + k) * nk + l) * nk + m;
                    int in = k + l + m <= L->P;
                    Uo[o] = in ? U[v][k][l][m] : 0.0;
                    Fo[o] = in ? F[v][k][l][m] : 0.0;
                    Go[o] = in ? G[v][k][l][m] : 0.0;
                }
}

double oracle2d_smoothness(const double* c, int n) { return o2_smoothness(c, n); }

/* Cells per axis of the stage produced from a stage of n_old cells. */
long oracle2d_new_count(const o2_law* L, int parity, long n_old) {
    if (L->bc == O2_PERIODIC) return n_old;
    return parity == 0 ? n_old - 1 : n_old + 1;
}

static long o2_parent_index(const o2_law* L, long j, long n_old) {
    if (L->bc == O2_PERIODIC) return ((j % n_old) + n_old) % n_old;
    if (j < 0) return 0;
    if (j > n_old - 1) return n_old - 1;
    return j;
}

/* One half-step over a whole stage old[ny_old][nx_old][nv][nq] (Sec. 3.1,
 * Fig. 2DMesh).  Writes new[ny_new][nx_new][nv][nq]; returns the number of
 * new cells, or -1 on bad arguments.  weights (may be NULL) receives
 * [cell][nv][5]. */
long oracle2d_halfstep(const o2_law* L, int parity, long nx_old, long ny_old, const double* old, double* out,
                       double lamx, double lamy, double* weights) {
    const int nv = o2_nv(L), nq = o2_nq(L->P), nd = nv * nq;
    if (L->P < 1 || L->P > O2_MAXP || nx_old < 2 || ny_old < 2) return -1;
    const long nx_new = oracle2d_new_count(L, parity, nx_old), ny_new = oracle2d_new_count(L, parity, ny_old);
    const long n_old = nx_old * ny_old;
    o2_parent* terms = (o2_parent*)malloc((size_t)n_old * sizeof(o2_parent));
    if (!terms) return -1;
    long c;
#pragma omp parallel for schedule(static)
    for (c = 0; c < n_old; ++c) o2_parent_terms(L, old + c * nd, lamx, lamy, &terms[c]);
#pragma omp parallel for schedule(static)
    for (c = 0; c < nx_new * ny_new; ++c) {
        long i = c % nx_new, j = c / nx_new;
        long il = parity == 0 ? i : i - 1, jl = parity == 0 ? j : j - 1;
        long x0 = o2_parent_index(L, il, nx_old), x1 = o2_parent_index(L, il + 1, nx_old);
        long y0 = o2_parent_index(L, jl, ny_old), y1 = o2_parent_index(L, jl + 1, ny_old);
        const o2_parent* pv[4] = {&terms[y0 * nx_old + x0], &terms[y0 * nx_old + x1], &terms[y1 * nx_old + x1],
                                  &terms[y1 * nx_old + x0]};
        o2_new_cell_from(L, pv, lamx, lamy, out + c * nd, weights ? weights + c * nv * 5 : NULL, NULL, NULL);
    }
    free(terms);
    return nx_new * ny_new;
}

/* Largest characteristic speeds over the centre point values of a stage:
 * out[0] = max |a_x| (advection), |u| (Burgers) or |u| + c (Euler) along x,
 * out[1] the same along y, out[2] = max over cells of sx/dx + sy/dy.  The
 * paper does not say how the 2D CFL bound is formed; the callers choose. */
void oracle2d_max_speeds(const o2_law* L, long n, const double* q, double dx, double dy, double* out) {
    const int nv = o2_nv(L), nq = o2_nq(L->P);
    double mx = 0.0, my = 0.0, ms = 0.0;
    for (long i = 0; i < n; ++i) {
        const double* c = q + i * nv * nq;
        double sx, sy;
        if (L->system == O2_ADVECTION) {
            sx = fabs(L->ax);
            sy = fabs(L->ay);
        } else if (L->system == O2_BURGERS) {
            sx = sy = fabs(c[0]);
        } else {
            double rho = c[0], u = c[nq] / rho, v = c[2 * nq] / rho, E = c[3 * nq];
            double p = (L->gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
            double a = sqrt(L->gamma * p / rho);
            sx = fabs(u) + a;
            sy = fabs(v) + a;
        }
        double s = sx / dx + sy / dy;
        if (sx > mx || sx != sx) mx = sx;
        if (sy > my || sy != sy) my = sy;
        if (s > ms || s != s) ms = s;
    }
    out[0] = mx;
    out[1] = my;
    out[2] = ms;
}
