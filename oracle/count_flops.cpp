// count_flops.cpp -- floating-point operation count of the oracle's 1D
// half-step (TEST INFRASTRUCTURE ONLY, like the rest of oracle/).
//
// wcc_oracle.c is compiled a second time, as C++, with `double` replaced by
// the counting type `cnt` below; its source is not changed.  A cnt carries
// its value and a flag telling whether it depends on the cell data (the
// DOFs and lam).  An arithmetic operation is counted when at least one
// operand depends on the data, so the binomial coefficients, factorials and
// powers of two the oracle recomputes from integers are not counted: the
// count is the work of the scheme as the oracle writes it (Sec. 2.1, 2.2,
// Sec. 4), with its formulation (derivative form, binomial Leibniz sums,
// divisions by constants, a numerical 3x3 inverse for the characteristic
// basis).
//
// Build and run: oracle/count_flops.py (g++ -x c++ -include this file's
// counting header part, see COUNT_FLOPS_HEADER below).
#ifndef COUNT_FLOPS_HEADER
#define COUNT_FLOPS_HEADER
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct Counts {
    long long add = 0, mul = 0, div = 0, sqrt = 0, pow = 0, cmp = 0;
};
static Counts g_counts;

struct cnt {
    double v;
    bool d;  // depends on the data
    cnt() : v(0.0), d(false) {}
    cnt(double x) : v(x), d(false) {}
    cnt(int x) : v((double)x), d(false) {}
    cnt(long x) : v((double)x), d(false) {}
    cnt(double x, bool dep) : v(x), d(dep) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
};

static inline cnt cnt_op(double r, const cnt& a, const cnt& b, long long& counter) {
    const bool dep = a.d || b.d;
    if (dep) ++counter;
    return cnt(r, dep);
}
static inline cnt operator+(const cnt& a, const cnt& b) { return cnt_op(a.v + b.v, a, b, g_counts.add); }
static inline cnt operator-(const cnt& a, const cnt& b) { return cnt_op(a.v - b.v, a, b, g_counts.add); }
static inline cnt operator*(const cnt& a, const cnt& b) { return cnt_op(a.v * b.v, a, b, g_counts.mul); }
static inline cnt operator/(const cnt& a, const cnt& b) { return cnt_op(a.v / b.v, a, b, g_counts.div); }
static inline cnt operator-(const cnt& a) { return cnt(-a.v, a.d); }
static inline cnt& operator+=(cnt& a, const cnt& b) { return a = a + b; }
static inline cnt& operator-=(cnt& a, const cnt& b) { return a = a - b; }
static inline cnt& operator*=(cnt& a, const cnt& b) { return a = a * b; }
static inline cnt& operator/=(cnt& a, const cnt& b) { return a = a / b; }
static inline bool cmp_count(const cnt& a, const cnt& b) {
    if (a.d || b.d) ++g_counts.cmp;
    return true;
}
static inline bool operator<(const cnt& a, const cnt& b) { return cmp_count(a, b) && a.v < b.v; }
static inline bool operator>(const cnt& a, const cnt& b) { return cmp_count(a, b) && a.v > b.v; }
static inline bool operator<=(const cnt& a, const cnt& b) { return cmp_count(a, b) && a.v <= b.v; }
static inline bool operator>=(const cnt& a, const cnt& b) { return cmp_count(a, b) && a.v >= b.v; }
static inline bool operator==(const cnt& a, const cnt& b) { return a.v == b.v; }
static inline bool operator!=(const cnt& a, const cnt& b) { return a.v != b.v; }
static inline cnt sqrt(const cnt& a) {
    if (a.d) ++g_counts.sqrt;
    return cnt(std::sqrt(a.v), a.d);
}
static inline cnt fabs(const cnt& a) { return cnt(std::fabs(a.v), a.d); }
static inline cnt pow(const cnt& a, const cnt& b) {
    const bool dep = a.d || b.d;
    if (dep) ++g_counts.pow;
    return cnt(std::pow(a.v, b.v), dep);
}
static inline cnt ldexp(const cnt& a, int e) { return cnt(std::ldexp(a.v, e), a.d); }

#define double cnt
#else  // the driver, compiled after wcc_oracle.c in the same translation unit
#undef double

// One half-step of a Euler / Burgers stage of smooth, non-trivial data; the
// flops per new cell of oracle_new_cell, and of one Cauchy-Kovalewski table
// (oracle_ck_table), which oracle_new_cell runs twice (once per parent,
// without reuse) while the scheme needs it once per parent.
int main(int argc, char** argv) {
    const int system = argc > 1 ? atoi(argv[1]) : OR_EULER;
    const int P = argc > 2 ? atoi(argv[2]) : 3;
    const int limiter = argc > 3 ? atoi(argv[3]) : 1;
    or_law L;
    L.system = system;
    L.P = P;
    L.limiter = limiter;
    L.bc = OR_PERIODIC;
    L.a = 1.0;
    L.gamma = 1.4;
    L.alpha = 2.0;
    L.eps = 1e-40;
    const int nv = system == OR_EULER ? 3 : 1, nk = P + 1;
    const int cells = 64;
    cnt* q = new cnt[cells * nv * nk];
    cnt* out = new cnt[cells * nv * nk];
    const double dx = 1.0 / cells;
    for (int i = 0; i < cells; ++i) {
        const double x = (i + 0.5) * dx, w = 2.0 * M_PI;
        for (int v = 0; v < nv; ++v)
            for (int k = 0; k <= P; ++k) {
                // rho = 1 + 0.2 sin, u = 0.5 + 0.1 cos, p = 1 + 0.1 sin (conserved
                // values only matter through the branches; any smooth data do)
                double base = (v == 0 ? 1.0 : v == 1 ? 0.5 : 2.6) + (system == OR_EULER ? 0.0 : -0.5);
                double amp = 0.2 / (v + 1);
                double val = (k == 0) ? base + amp * std::sin(w * x)
                                      : amp * std::pow(w * dx, k) * std::sin(w * x + k * M_PI / 2);
                q[(i * nv + v) * nk + k] = cnt(val, true);
            }
    }
    const cnt lam(0.2 / 2.2, true);
    g_counts = Counts();
    oracle_halfstep(&L, 0, cells, q, out, lam, NULL);
    const Counts all = g_counts;
    g_counts = Counts();
    cnt U[OR_MAXV * OR_NK * OR_NK], F[OR_MAXV * OR_NK * OR_NK];
    oracle_ck_table(&L, q, lam, U, F);
    const Counts ck = g_counts;
    auto per = [&](long long x) { return (double)x / cells; };
    // per cell-update: everything once, minus the second (redundant) CK table
    printf("{\"system\": %d, \"P\": %d, \"limiter\": %d, \"per_new_cell_as_written\": "
           "{\"add\": %.1f, \"mul\": %.1f, \"div\": %.1f, \"sqrt\": %.1f, \"pow\": %.1f, \"cmp\": %.1f}, "
           "\"ck_table\": {\"add\": %lld, \"mul\": %lld, \"div\": %lld, \"sqrt\": %lld, \"pow\": %lld}, "
           "\"per_cell_update\": {\"add\": %.1f, \"mul\": %.1f, \"div\": %.1f, \"sqrt\": %.1f, \"pow\": %.1f}}\n",
           system, P, limiter, per(all.add), per(all.mul), per(all.div), per(all.sqrt), per(all.pow), per(all.cmp),
           ck.add, ck.mul, ck.div, ck.sqrt, ck.pow, per(all.add) - ck.add, per(all.mul) - ck.mul,
           per(all.div) - ck.div, per(all.sqrt) - ck.sqrt, per(all.pow) - ck.pow);
    delete[] q;
    delete[] out;
    return 0;
}
#endif
