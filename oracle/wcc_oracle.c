/*
 * wcc_oracle.c -- plain, slow FP64 CPU oracle for the 1D weighted compact
 * central (WCC) half-step of Shen & Parsani, "A class of high-order weighted
 * compact central schemes for solving hyperbolic conservation laws"
 * (arXiv 2104.04347).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  The
 * product path (the CUDA library) shares no code, header, table or helper
 * with it.
 *
 * Conventions (all from Sec. 2.1 of the paper):
 *   - DOFs are the paper's scaled derivatives u_kx = dx^k d^k u/dx^k at the
 *     cell centre (Eq. 1D_Derivative_DEF, Eq. 1DPolynomial_Space), stored
 *     [cell][var][k] with k = 0..P.
 *   - dt is the HALF step t^{n+1/2} - t^n (Eq. 1DFlux), lam = dt/dx.
 *   - Parity 0 advances an integer stage to the half stage: new[i] is the
 *     staggered cell [x_i, x_{i+1}] built from old[i] (left) and old[i+1]
 *     (right).  Parity 1 advances a half stage to the integer stage:
 *     new[i] is built from old[i-1] and old[i].
 *   - Periodic: both stages hold N cells.  Transmissive: the integer stage
 *     holds N+1 cells centred on the grid points x_L + i dx, the half stage
 *     N cells; the ghost staggered cells x_{1/2}, x_{N+3/2} are copies of the
 *     adjacent cell's DOFs (zeroth-order extrapolation).
 *
 * Written for readability, not speed: binomial-coefficient (Leibniz) sums in
 * the paper's derivative form, no blocking, no fusion, no reuse of a parent's
 * Cauchy-Kovalewski result between its two children.  Compiled with
 * -O2 -ffp-contract=off so that every product and sum is rounded as written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXP 6
#define OR_MAXV 3
#define OR_NK (OR_MAXP + 1)

enum { OR_ADVECTION = 0, OR_BURGERS = 1, OR_EULER = 2 };
enum { OR_PERIODIC = 0, OR_TRANSMISSIVE = 1 };

/* The conservation law and scheme options.  Field order is part of the
 * ctypes interface in oracle/__init__.py. */
typedef struct {
    int system;    /* OR_ADVECTION (f = a u), OR_BURGERS (f = u^2/2), OR_EULER */
    int P;         /* polynomial degree, 0..4 */
    int limiter;   /* 1: WENO-type limiter of Sec. 2.2 on every new cell */
    int bc;        /* OR_PERIODIC or OR_TRANSMISSIVE */
    double a;      /* advection speed */
    double gamma;  /* ratio of specific heats (Euler) */
    double alpha;  /* weight exponent (Eq. 1D2ndOrderWeights / 1DHighOrderWeights) */
    double eps;    /* epsilon in the weights, 1e-40 in the paper */
} or_law;

static int or_nv(const or_law* L) { return L->system == OR_EULER ? 3 : 1; }

static double or_fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

static double or_binom(int n, int k) {
    return or_fact(n) / (or_fact(k) * or_fact(n - k));
}

static double or_pow2(int n) { return ldexp(1.0, n); }

/* Scaled derivative arrays X[a][b] = dx^a dt^b d^a_x d^b_t X at the cell
 * centre, time level t^n, for a + b <= P. */
typedef double or_series[OR_NK][OR_NK];

/* Generalised Leibniz rule for the product Z = X Y, entry (a, b):
 * Z_ab = sum_{i<=a, j<=b} C(a,i) C(b,j) X_ij Y_{a-i,b-j}.  The scaling by
 * dx^a dt^b distributes over the two factors, so the rule holds as written
 * for the scaled arrays (Sec. 4, Dyson / Dumbser-Munz). */
static double or_leibniz(or_series X, or_series Y, int a, int b) {
    double s = 0.0;
    for (int i = 0; i <= a; ++i)
        for (int j = 0; j <= b; ++j)
            s += or_binom(a, i) * or_binom(b, j) * X[i][j] * Y[a - i][b - j];
    return s;
}

/* Cauchy-Kovalewski procedure (Eq. 1DCauchy_Kovalewski, Sec. 4 for systems).
 * In scaled form the PDE u_t = -f_x reads U_{a,b+1} = -lam F_{a+1,b}.
 * Level b = 0 holds the stored DOFs; at each level the flux derivatives
 * F_{a,b} (a <= P-b) follow from the chain / Leibniz rule, and then give the
 * next level of U.  On return U and F hold every entry with a + b <= P. */
static void or_cauchy_kovalewski(const or_law* L, const double* q, double lam,
                                 or_series U[OR_MAXV], or_series F[OR_MAXV]) {
    const int P = L->P, nv = or_nv(L);
    or_series w, qq, p, Ep; /* Euler auxiliaries: velocity, rho u^2, pressure, E + p */
    memset(w, 0, sizeof(w));
    memset(qq, 0, sizeof(qq));
    memset(p, 0, sizeof(p));
    memset(Ep, 0, sizeof(Ep));
    for (int v = 0; v < nv; ++v) {
        memset(U[v], 0, sizeof(or_series));
        memset(F[v], 0, sizeof(or_series));
        for (int a = 0; a <= P; ++a) U[v][a][0] = q[v * (P + 1) + a];
    }
    for (int b = 0; b <= P; ++b) {
        for (int a = 0; a <= P - b; ++a) {
            if (L->system == OR_ADVECTION) {
                F[0][a][b] = L->a * U[0][a][b];
            } else if (L->system == OR_BURGERS) {
                F[0][a][b] = 0.5 * or_leibniz(U[0], U[0], a, b);
            } else {
                /* U = (rho, m, E).  Velocity w from m = rho w:
                 * m_ab = sum C C rho_ij w_{a-i,b-j}, solved for w_ab. */
                double s = U[1][a][b];
                for (int i = 0; i <= a; ++i)
                    for (int j = 0; j <= b; ++j) {
                        if (i == 0 && j == 0) continue;
                        s -= or_binom(a, i) * or_binom(b, j) * U[0][i][j] * w[a - i][b - j];
                    }
                w[a][b] = s / U[0][0][0];
                qq[a][b] = or_leibniz(U[1], w, a, b);              /* rho u^2 */
                p[a][b] = (L->gamma - 1.0) * (U[2][a][b] - 0.5 * qq[a][b]);
                Ep[a][b] = U[2][a][b] + p[a][b];
                F[0][a][b] = U[1][a][b];                            /* rho u */
                F[1][a][b] = qq[a][b] + p[a][b];                    /* rho u^2 + p */
                F[2][a][b] = or_leibniz(Ep, w, a, b);               /* (E + p) u */
            }
        }
        if (b < P)
            for (int a = 0; a <= P - b - 1; ++a)
                for (int v = 0; v < nv; ++v) U[v][a][b + 1] = -lam * F[v][a + 1][b];
    }
}

/* Smoothness indicator of a degree-n polynomial with scaled derivatives
 * c[0..n] (Eq. 1DSmoothIndicator).  With xi = (x - x_i)/dx the factors of
 * dx cancel and beta = sum_{k=1}^{n} int_{-1/2}^{1/2} (d^k u/dxi^k)^2 dxi,
 * where d^k u/dxi^k = sum_{j>=k} c_j xi^{j-k}/(j-k)!.  The square is
 * expanded term by term with int xi^e dxi = 1/((e+1) 2^e) for even e, 0 for
 * odd e. */
static double or_smoothness(const double* c, int n) {
    double beta = 0.0;
    for (int k = 1; k <= n; ++k)
        for (int j = k; j <= n; ++j)
            for (int l = k; l <= n; ++l) {
                int e = (j - k) + (l - k);
                if (e % 2) continue;
                double moment = 1.0 / ((double)(e + 1) * or_pow2(e));
                beta += c[j] * c[l] / (or_fact(j - k) * or_fact(l - k)) * moment;
            }
    return beta;
}

/* Value of the polynomial of Eq. 1DPolynomial_Space at xi. */
static double or_poly_value(const double* c, int n, double xi) {
    double s = 0.0;
    for (int k = 0; k <= n; ++k) s += c[k] * pow(xi, (double)k) / or_fact(k);
    return s;
}

/* Limiter for one scalar component (Sec. 2.2).
 * d[0..P]: DOFs of u_0 (Eq. 1DU0), overwritten with those of u_*;
 * ubar: cell average of u_0; vl, vr: time-extrapolated vertex values
 * u_{i-1/2}, u_{i+1/2} (Eq. SubEq:Cal_1D_Derivatives_4).
 * wout (may be NULL) receives w_0, w_1, w_2. */
static void or_limit_scalar(const or_law* L, double* d, double ubar, double vl, double vr,
                            double* wout) {
    const int P = L->P;
    /* Two linear candidates (Eq. 1DU12): mean ubar, one-sided slopes. */
    double c1[2] = {ubar, 2.0 * (ubar - vl)};
    double c2[2] = {ubar, 2.0 * (vr - ubar)};
    double beta[3] = {or_smoothness(d, P), or_smoothness(c1, 1), or_smoothness(c2, 1)};
    double wh[3];
    if (P == 1) {
        /* Eq. 1D2ndOrderWeights */
        for (int m = 0; m < 3; ++m) wh[m] = pow(1.0 / (beta[m] + L->eps), L->alpha);
    } else {
        /* Eq. 1DHighOrderWeights: sigma = residuals between the space
         * polynomial and the time-extrapolated vertex values; tau = smoothness
         * of the highest-order term. */
        double rr = or_poly_value(d, P, 0.5) - vr;
        double rl = or_poly_value(d, P, -0.5) - vl;
        double sigma = rr * rr + rl * rl;
        double tau = d[P] * d[P];
        for (int m = 0; m < 3; ++m)
            wh[m] = pow(sigma * tau / (beta[m] * beta[m] + L->eps), L->alpha);
        wh[0] += 1.0;
    }
    double sum = wh[0] + wh[1] + wh[2];
    double w[3] = {wh[0] / sum, wh[1] / sum, wh[2] / sum};
    /* Eq. 1DLimitedPolynomial: u_* = w0 u_0 + w1 u_1 + w2 u_2, DOF by DOF. */
    double limited[OR_NK];
    limited[0] = w[0] * d[0] + w[1] * c1[0] + w[2] * c2[0];
    if (P >= 1) limited[1] = w[0] * d[1] + w[1] * c1[1] + w[2] * c2[1];
    for (int k = 2; k <= P; ++k) limited[k] = w[0] * d[k];
    for (int k = 0; k <= P; ++k) d[k] = limited[k];
    if (wout) {
        wout[0] = w[0];
        wout[1] = w[1];
        wout[2] = w[2];
    }
}

/* Solve R X = I for the 3x3 inverse by Gauss-Jordan elimination with partial
 * pivoting (plain textbook method). */
static void or_invert3(double R[3][3], double Linv[3][3]) {
    double A[3][6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = R[i][j];
            A[i][3 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 6; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        double inv = 1.0 / A[c][c];
        for (int j = 0; j < 6; ++j) A[c][j] *= inv;
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            double f = A[r][c];
            for (int j = 0; j < 6; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Linv[i][j] = A[i][3 + j];
}

/* Right eigenvectors of the Euler flux Jacobian A(U) in conserved variables
 * (columns for u-c, u, u+c; Toro's textbook form, cited in Sec. 5.2), and the
 * left eigenvectors as the matrix inverse.  Exposed for tests. */
void oracle_euler_eigenvectors(double gamma, const double* U, double* Rout, double* Lout) {
    double rho = U[0], u = U[1] / U[0], E = U[2];
    double p = (gamma - 1.0) * (E - 0.5 * rho * u * u);
    double c = sqrt(gamma * p / rho);
    double H = (E + p) / rho;
    double R[3][3] = {{1.0, 1.0, 1.0}, {u - c, u, u + c}, {H - u * c, 0.5 * u * u, H + u * c}};
    double Li[3][3];
    or_invert3(R, Li);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Rout[3 * i + j] = R[i][j];
            Lout[3 * i + j] = Li[i][j];
        }
}

/* One new staggered cell from its left parent qL and right parent qR
 * (each nv*(P+1) DOFs, [var][k]).  Writes the new DOFs to out.  Optional
 * diagnostics: cand[3][nv][P+1] receives u_0, u_1, u_2 as DOF vectors before
 * limiting (u_1, u_2 padded with zeros), weights[nv][3] the limiter weights
 * (per characteristic component for Euler), ubar_out[nv] the new cell
 * average. */
void oracle_new_cell(const or_law* L, const double* qL, const double* qR, double lam,
                     double* out, double* cand, double* weights, double* ubar_out) {
    const int P = L->P, nv = or_nv(L), nk = P + 1;
    or_series UL[OR_MAXV], FL[OR_MAXV], UR[OR_MAXV], FR[OR_MAXV];
    or_cauchy_kovalewski(L, qL, lam, UL, FL);
    or_cauchy_kovalewski(L, qR, lam, UR, FR);

    double d[OR_MAXV][OR_NK], ubar[OR_MAXV], vl[OR_MAXV], vr[OR_MAXV];
    for (int v = 0; v < nv; ++v) {
        /* Eq. Cal1DFlux: time-averaged flux at each vertex. */
        double fbarL = 0.0, fbarR = 0.0;
        for (int k = 0; k <= P; ++k) {
            fbarL += FL[v][0][k] / or_fact(k + 1);
            fbarR += FR[v][0][k] / or_fact(k + 1);
        }
        /* Eqs. SubEq:1DCellAVGR, SubEq:1DCellAVGL: half-cell averages. */
        double ubarR = 0.0, ubarL = 0.0;
        for (int k = 0; k <= P; ++k) {
            double coef = 1.0 / (or_fact(k + 1) * or_pow2(k));
            ubarR += coef * qL[v * nk + k];
            ubarL += ((k % 2) ? -coef : coef) * qR[v * nk + k];
        }
        /* Eq. SubEq:1DIntegral: finite-volume update of the cell average. */
        ubar[v] = 0.5 * (ubarR + ubarL) + lam * (fbarL - fbarR);

        /* Eq. SubEq:Cal_1D_Derivatives_4: vertex values at t^{n+1/2}. */
        double VL[OR_NK], VR[OR_NK];
        for (int k = 0; k <= P; ++k) {
            VL[k] = 0.0;
            VR[k] = 0.0;
            for (int m = 0; m <= P - k; ++m) {
                VL[k] += UL[v][k][m] / or_fact(m);
                VR[k] += UR[v][k][m] / or_fact(m);
            }
        }
        vl[v] = VL[0];
        vr[v] = VR[0];
        /* Eq. SubEq:Cal_1D_Derivatives_3: derivatives from high to low order. */
        for (int k = P - 1; k >= 0; --k) {
            double s = VR[k] - VL[k];
            for (int m = 3; m <= P - k; ++m) {
                double coef = (1.0 - ((m % 2) ? -1.0 : 1.0)) / (or_fact(m) * or_pow2(m));
                s -= coef * d[v][k + m];
            }
            d[v][k + 1] = s;
        }
        /* Eq. 1DCalU: the point value from the cell average. */
        double s = ubar[v];
        for (int k = 2; k <= P; ++k) {
            double coef = (1.0 + ((k % 2) ? -1.0 : 1.0)) / (or_fact(k + 1) * or_pow2(k + 1));
            s -= coef * d[v][k];
        }
        d[v][0] = s;
    }

    if (cand) {
        for (int i = 0; i < 3 * nv * nk; ++i) cand[i] = 0.0;
        for (int v = 0; v < nv; ++v) {
            for (int k = 0; k <= P; ++k) cand[(0 * nv + v) * nk + k] = d[v][k];
            cand[(1 * nv + v) * nk + 0] = ubar[v];
            cand[(2 * nv + v) * nk + 0] = ubar[v];
            if (P >= 1) {
                cand[(1 * nv + v) * nk + 1] = 2.0 * (ubar[v] - vl[v]);
                cand[(2 * nv + v) * nk + 1] = 2.0 * (vr[v] - ubar[v]);
            }
        }
    }
    if (ubar_out)
        for (int v = 0; v < nv; ++v) ubar_out[v] = ubar[v];

    if (L->limiter && P >= 1) {
        if (nv == 1) {
            or_limit_scalar(L, d[0], ubar[0], vl[0], vr[0], weights);
        } else {
            /* Sec. 4: limit the characteristic variables L(ubar) U, then map
             * back with R(ubar). */
            double R[9], Lm[9];
            oracle_euler_eigenvectors(L->gamma, ubar, R, Lm);
            double cd[OR_MAXV][OR_NK], cub[OR_MAXV], cvl[OR_MAXV], cvr[OR_MAXV];
            for (int i = 0; i < 3; ++i) {
                cub[i] = cvl[i] = cvr[i] = 0.0;
                for (int k = 0; k <= P; ++k) cd[i][k] = 0.0;
                for (int j = 0; j < 3; ++j) {
                    cub[i] += Lm[3 * i + j] * ubar[j];
                    cvl[i] += Lm[3 * i + j] * vl[j];
                    cvr[i] += Lm[3 * i + j] * vr[j];
                    for (int k = 0; k <= P; ++k) cd[i][k] += Lm[3 * i + j] * d[j][k];
                }
            }
            for (int i = 0; i < 3; ++i)
                or_limit_scalar(L, cd[i], cub[i], cvl[i], cvr[i], weights ? weights + 3 * i : NULL);
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k <= P; ++k) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i) s += R[3 * j + i] * cd[i][k];
                    d[j][k] = s;
                }
        }
    }
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k <= P; ++k) out[v * nk + k] = d[v][k];
}

/* Number of cells of the stage produced from a stage of n_old cells. */
int oracle_new_count(const or_law* L, int parity, long n_old) {
    if (L->bc == OR_PERIODIC) return (int)n_old;
    return (int)(parity == 0 ? n_old - 1 : n_old + 1);
}

static long or_parent(const or_law* L, long j, long n_old) {
    if (L->bc == OR_PERIODIC) return ((j % n_old) + n_old) % n_old;
    if (j < 0) return 0;                   /* ghost x_{1/2}: copy of the first cell */
    if (j > n_old - 1) return n_old - 1;   /* ghost x_{N+3/2}: copy of the last cell */
    return j;
}

/* One half-step over a whole stage (Sec. 2.1, Fig. 1).  Returns the number
 * of new cells, or -1 on bad arguments.  weights (may be NULL) receives
 * [cell][nv][3] limiter weights. */
long oracle_halfstep(const or_law* L, int parity, long n_old, const double* old, double* out,
                     double lam, double* weights) {
    const int nv = or_nv(L), nq = nv * (L->P + 1);
    if (L->P < 0 || L->P > OR_MAXP || n_old < 2) return -1;
    long n_new = oracle_new_count(L, parity, n_old);
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n_new; ++i) {
        long jl = (parity == 0) ? i : i - 1;
        long pl = or_parent(L, jl, n_old), pr = or_parent(L, jl + 1, n_old);
        oracle_new_cell(L, old + pl * nq, old + pr * nq, lam, out + i * nq, NULL,
                        weights ? weights + i * nv * 3 : NULL, NULL);
    }
    return n_new;
}

/* Largest characteristic speed over the centre point values of a stage:
 * |a| (advection), |u| (Burgers), |u| + c (Euler).  The paper does not say
 * how the CFL bound is evaluated; this is the reading used throughout. */
double oracle_max_speed(const or_law* L, long n, const double* q) {
    const int nv = or_nv(L), nk = L->P + 1;
    double amax = 0.0;
    for (long i = 0; i < n; ++i) {
        double s;
        if (L->system == OR_ADVECTION) {
            s = fabs(L->a);
        } else if (L->system == OR_BURGERS) {
            s = fabs(q[i * nv * nk]);
        } else {
            double rho = q[i * nv * nk], m = q[i * nv * nk + nk], E = q[i * nv * nk + 2 * nk];
            double u = m / rho;
            double p = (L->gamma - 1.0) * (E - 0.5 * rho * u * u);
            s = fabs(u) + sqrt(L->gamma * p / rho);
        }
        if (s > amax || s != s) amax = s;
    }
    return amax;
}

/* Scaled Cauchy-Kovalewski table of one cell, exposed for tests:
 * U_out, F_out are [nv][P+1][P+1] with entry (a, b) = dx^a dt^b d_x^a d_t^b. */
void oracle_ck_table(const or_law* L, const double* q, double lam, double* U_out, double* F_out) {
    const int nv = or_nv(L), nk = L->P + 1;
    or_series U[OR_MAXV], F[OR_MAXV];
    or_cauchy_kovalewski(L, q, lam, U, F);
    for (int v = 0; v < nv; ++v)
        for (int a = 0; a < nk; ++a)
            for (int b = 0; b < nk; ++b) {
                U_out[(v * nk + a) * nk + b] = (a + b <= L->P) ? U[v][a][b] : 0.0;
                F_out[(v * nk + a) * nk + b] = (a + b <= L->P) ? F[v][a][b] : 0.0;
            }
}

/* Smoothness indicator exposed for tests. */
double oracle_smoothness(const double* c, int n) { return or_smoothness(c, n); }

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
