// wcc_stability.cu -- the library's own von Neumann analysis of the linear
// scheme (Sec. 2.3), host code: the CFL limit of each degree P and the
// default CFL number wcc_default_cfl picks from it.
//
// For linear advection u_t + u_x = 0 (speed 1, limiter off) one half-step is
// linear in the two parents' coefficients: new = M_L q_left + M_R q_right
// (Eq. 1DSchemeMatrixForm).  A Fourier mode of wavenumber theta per cell
// width sees the half-step amplification matrix
//     G(theta) = M_L e^{-i theta/2} + M_R e^{i theta/2}
// (Eq. 1DFourierAnalysis), and the scheme is stable for the CFL number nu
// when every eigenvalue of G(theta) lies in the closed unit disk for every
// theta (Eq. LinearStabilityCondition).  The limit is the largest such nu,
// found by bisection over a grid of theta.
//
// M_L, M_R are built here from the half-step in Taylor coefficients e_k =
// u_kx / k! (the form the kernels use; a diagonal change of basis, which
// leaves the eigenvalues unchanged): the Cauchy-Kovalewski table of each
// parent, the flux integral and half-cell averages, the new cell average,
// the vertex values and the derivatives from high to low order.
#include <cmath>
#include <complex>
#include <mutex>

#include "../../include/wcc.h"

namespace {

constexpr int kMaxP = 6;
constexpr int kMaxK = kMaxP + 1;
using cplx = std::complex<double>;

double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}
double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

// Parent record of linear advection with speed 1 at lam = dt/dx: the shares
// A (to the new cell on its right) and B (to the one on its left) of the cell
// average, and the vertex Taylor coefficients at the new time level.
void parent(int P, double lam, const double* c, double& A, double& B, double* vtx) {
    const int K = P + 1;
    double X[kMaxK][kMaxK] = {};
    for (int a = 0; a < K; ++a) X[a][0] = c[a];
    // u_t = -u_x in Taylor form: X[a][b+1] = -lam (a+1)/(b+1) X[a+1][b]
    for (int b = 0; b < P; ++b)
        for (int a = 0; a + b < P; ++a) X[a][b + 1] = -lam * (a + 1.0) / (b + 1.0) * X[a + 1][b];
    // Eq. Cal1DFlux: fbar = sum_b f[0][b] / (b + 1), f = u
    double fbar = 0.0;
    for (int b = 0; b < K; ++b) fbar += X[0][b] / (b + 1.0);
    // Eqs. SubEq:1DCellAVGR / SubEq:1DCellAVGL: half-cell averages
    double ur = 0.0, ul = 0.0;
    for (int k = 0; k < K; ++k) {
        const double w = 1.0 / ((k + 1.0) * std::ldexp(1.0, k));
        ur += w * c[k];
        ul += ((k & 1) ? -w : w) * c[k];
    }
    A = 0.5 * ur + lam * fbar;
    B = 0.5 * ul - lam * fbar;
    // Eq. SubEq:Cal_1D_Derivatives_4: vertex values at the new time level
    for (int k = 0; k < K; ++k) {
        vtx[k] = 0.0;
        for (int m = 0; m + k < K; ++m) vtx[k] += X[k][m];
    }
}

// One new cell from the left and right parents' coefficients.
void new_cell(int P, double lam, const double* cl, const double* cr, double* e) {
    double AL, BL, AR, BR, vL[kMaxK], vR[kMaxK];
    parent(P, lam, cl, AL, BL, vL);
    parent(P, lam, cr, AR, BR, vR);
    const double ubar = AL + BR;  // Eq. SubEq:1DIntegral
    // Eq. SubEq:Cal_1D_Derivatives_3 from the highest order down
    for (int k = P - 1; k >= 0; --k) {
        double s = vR[k] - vL[k];
        for (int m = 3; m <= P - k; m += 2) s -= 2.0 * binom(k + m, m) * std::ldexp(1.0, -m) * e[k + m];
        e[k + 1] = s / (k + 1.0);
    }
    // Eq. 1DCalU: centre value from the cell average
    double u0 = ubar;
    for (int k = 2; k <= P; k += 2) u0 -= e[k] / ((k + 1.0) * std::ldexp(1.0, k));
    e[0] = u0;
}

// Largest |eigenvalue| of the n x n complex matrix G: characteristic
// polynomial by the Faddeev-LeVerrier recursion, its roots by the
// Durand-Kerner iteration (warm-started from `roots`, updated in place).
double spectral_radius(int n, const cplx (*G)[kMaxK], cplx* roots) {
    cplx coef[kMaxK + 1];  // monic: coef[n] = 1
    cplx M[kMaxK][kMaxK] = {}, AM[kMaxK][kMaxK];
    coef[n] = 1.0;
    for (int k = 1; k <= n; ++k) {
        // M_k = G M_{k-1} + coef[n-k+1] I, coef[n-k] = -tr(G M_k) / k
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                cplx s = 0.0;
                for (int l = 0; l < n; ++l) s += G[i][l] * M[l][j];
                AM[i][j] = s;
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) M[i][j] = AM[i][j] + (i == j ? coef[n - k + 1] : cplx(0.0));
        cplx tr = 0.0;
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < n; ++l) tr += G[i][l] * M[l][i];
        coef[n - k] = -tr / double(k);
    }
    auto poly = [&](cplx z) {
        cplx p = coef[n];
        for (int k = n - 1; k >= 0; --k) p = p * z + coef[k];
        return p;
    };
    for (int it = 0; it < 500; ++it) {
        double change = 0.0;
        for (int i = 0; i < n; ++i) {
            cplx den = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= roots[i] - roots[j];
            if (std::abs(den) == 0.0) den = 1e-300;
            const cplx step = poly(roots[i]) / den;
            roots[i] -= step;
            change = std::fmax(change, std::abs(step));
        }
        if (change < 1e-15) break;
    }
    double r = 0.0;
    for (int i = 0; i < n; ++i) r = std::fmax(r, std::abs(roots[i]));
    return r;
}

constexpr int kThetas = 2048;

// max over theta of the spectral radius of G(theta) at CFL nu.
double max_radius(int P, double nu) {
    const int K = P + 1;
    double ML[kMaxK][kMaxK], MR[kMaxK][kMaxK];
    for (int j = 0; j < K; ++j) {
        double unit[kMaxK] = {}, zero[kMaxK] = {}, e[kMaxK];
        unit[j] = 1.0;
        new_cell(P, nu, unit, zero, e);
        for (int i = 0; i < K; ++i) ML[i][j] = e[i];
        new_cell(P, nu, zero, unit, e);
        for (int i = 0; i < K; ++i) MR[i][j] = e[i];
    }
    cplx roots[kMaxK];
    for (int i = 0; i < K; ++i) roots[i] = std::pow(cplx(0.4, 0.9), i + 1);
    double worst = 0.0;
    const double pi = std::acos(-1.0);
    for (int m = 1; m < kThetas; ++m) {
        const double th = 2.0 * pi * m / kThetas;
        const cplx em = std::polar(1.0, -0.5 * th), ep = std::polar(1.0, 0.5 * th);
        cplx G[kMaxK][kMaxK];
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) G[i][j] = ML[i][j] * em + MR[i][j] * ep;
        worst = std::fmax(worst, spectral_radius(K, G, roots));
    }
    return worst;
}

// Largest nu in (0, 1] with max radius <= 1 + 1e-9, by bisection (the
// stable set is an interval from 0, which the scan confirms at every P).
double compute_limit(int P) {
    double lo = 1e-3, hi = 1.0;
    if (max_radius(P, lo) > 1.0 + 1e-9) return 0.0;
    for (int it = 0; it < 40; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (max_radius(P, mid) <= 1.0 + 1e-9)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

std::mutex g_mutex;
double g_limit[kMaxP + 1] = {};

}  // namespace

extern "C" int wcc_stability_limit(int P, double* nu) {
    if (P < 1 || P > kMaxP || !nu) return WCC_E_INVAL;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_limit[P] == 0.0) g_limit[P] = compute_limit(P);
    *nu = g_limit[P];
    return WCC_OK;
}

extern "C" int wcc_default_cfl(int P, double* cfl) {
    if (P < 1 || P > kMaxP || !cfl) return WCC_E_INVAL;
    // Sec. 5 runs P = 1, 2, 3 at nu = 0.4, 0.3, 0.25; above that the paper
    // gives no number, and the default is 0.8 of the degree's limit, rounded
    // down to two digits
    static const double paper[4] = {0.0, 0.4, 0.3, 0.25};
    if (P <= 3) {
        *cfl = paper[P];
        return WCC_OK;
    }
    double lim = 0.0;
    const int rc = wcc_stability_limit(P, &lim);
    if (rc != WCC_OK) return rc;
    *cfl = std::floor(80.0 * lim) / 100.0;
    return WCC_OK;
}
