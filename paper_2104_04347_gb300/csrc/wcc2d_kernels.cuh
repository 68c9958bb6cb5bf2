// wcc2d_kernels.cuh -- kernels of the 2D WCC path: the fused half-step, the
// CFL rate of a loaded stage, and the conversions between the host layout
// [row][col][var][q] (FP64) and the device planes.
//
// Device layout: plane (v, q) holds u_{kx,ly} of variable v (q = position of
// (k, l)) for every cell, row-major with `pitch` elements per row; planes are
// `plane` elements apart.  T is double (FP64 path) or float (FP32 path).
//
// The half-step kernel runs one CTA of TW threads per strip of TW - 1 new
// columns and `rows_per_cta` new rows.  It marches up the strip: each step
// computes the Cauchy-Kovalewski expansion and Appendix-B terms of one row of
// TW parents (thread t: parent column t of the strip) into a two-row ring
// in shared memory; the new cells between the previous parent row and this
// one then read their four parents from the ring (thread t: new cell between
// parent columns t and t + 1).  Every parent is expanded once per strip; the
// first parent row of a strip is also expanded by the strip below.
#pragma once

#include <algorithm>

#include "wcc2d_scheme.cuh"

namespace wcc2d {

struct DevState2D {
    // rate_bits[s]: max over the stage of parity s of s_x/dx + s_y/dy at
    // the cell centres, as the bit pattern of a non-negative double
    unsigned long long rate_bits[2];
    double t;
    long long step;
    unsigned int blocks_done;
    unsigned int err;  // ERR_* bits, sticky
};

struct Step2D {
    const void* in;
    void* out;
    long long pitch, plane;
    long long rows_alloc;  // rows of a plane
    int nx_old, ny_old, nx_new, ny_new;
    int parity, bc, rows_per_cta;
    double dx, dy;
    double inv_dx, inv_dy;  // 1 / dx, 1 / dy (host)
    double dt_given;  // > 0: the half-step size; otherwise cfl / rate of the old stage
    double cfl;
    Law2D law;
    DevState2D* st;
    double* hist;
    long long hist_cap;
};

__device__ __forceinline__ int parent_index(int j, int n_old, int bc) {
    if (bc == PERIODIC) {
        // one wrap covers every index a strip touches on meshes wider than
        // the strip; the remainder is for the narrow ones
        if (j >= -n_old && j < 2 * n_old) return j < 0 ? j + n_old : (j >= n_old ? j - n_old : j);
        j %= n_old;
        return j < 0 ? j + n_old : j;
    }
    return j < 0 ? 0 : (j > n_old - 1 ? n_old - 1 : j);
}

// Reads parent records from the ring: vertex r = 0..3 is parent column t
// (r = 0, 3) or t + 1 (r = 1, 2) of the lower (r = 0, 1) or upper row.
template <class T, int TW, int NV, int NQ1>
struct RingReader {
    const T* lo;
    const T* hi;
    int t;
    __device__ __forceinline__ T get(int r, int f) const {
        return r == 0 ? lo[f * TW + t] : r == 1 ? lo[f * TW + t + 1] : r == 2 ? hi[f * TW + t + 1] : hi[f * TW + t];
    }
    __device__ __forceinline__ T c(int r, int v) const { return get(r, v * 4 + r); }
    __device__ __forceinline__ T V(int r, int v, int q) const { return get(r, NV * 4 + v * NQ1 + q); }
};

template <int SYS, int P>
__host__ __device__ constexpr int record_fields() {
    return nvars(SYS) * (4 + nq(P - 1));
}

template <class T, int TW>
__host__ __device__ constexpr size_t ring_bytes(int fields) {
    return 2 * (size_t)fields * TW * sizeof(T);
}

// The half-step size: dt_given, or cfl over the rate of the old stage.  One
// thread takes the FP64 division and shares it (block barrier).
__device__ __forceinline__ double step_dt2d(const Step2D& a) {
    __shared__ double s_dt;
    if (threadIdx.x == 0) {
        double dt = a.dt_given;
        if (!(dt > 0.0)) dt = a.cfl / __longlong_as_double((long long)a.st->rate_bits[a.parity]);
        s_dt = dt;
    }
    __syncthreads();
    return s_dt;
}

// Block-wide max of the rate and OR of the error bits, one atomic each per
// CTA; the CTA that finishes last does the half-step's bookkeeping.
template <class T, int NT>
__device__ __forceinline__ void finish2d(T rate, unsigned err, double dt, const Step2D& a) {
    __shared__ double s_max[NT / 32];
    __shared__ unsigned s_err[NT / 32];
    double r = (double)rate;
    if (r != r) {
        r = INFINITY;
        err |= ERR_NONFINITE;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
        s_max[threadIdx.x >> 5] = r;
        s_err[threadIdx.x >> 5] = err;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = s_max[0];
        unsigned e = s_err[0];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w) {
            m = fmax(m, s_max[w]);
            e |= s_err[w];
        }
        DevState2D* st = a.st;
        atomicMax(&st->rate_bits[a.parity ^ 1], (unsigned long long)__double_as_longlong(m));
        if (e) atomicOr(&st->err, e);
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y;
        const unsigned done = atomicAdd(&st->blocks_done, 1u);
        if (done == total - 1) {
            __threadfence();
            // every CTA has read rate_bits[parity]; clear it for the launch after next
            st->rate_bits[a.parity] = 0ull;
            const long long k = st->step;
            if (k < a.hist_cap) a.hist[k] = dt;
            st->step = k + 1;
            st->t = st->t + dt;
            st->blocks_done = 0u;
            if (!(dt > 0.0) || dt == INFINITY) st->err |= ERR_NONFINITE;
            __threadfence();
        }
    }
}

// Resident CTAs the FP32 kernels are compiled for (caps their registers at
// 65536 / (4 x TW)); FP64 kernels are bound by the FP64 pipe and keep their
// registers.
template <class T>
constexpr int min_ctas2d() {
    return sizeof(T) == 4 ? 4 : 1;
}

template <int SYS, int P, class T, int TW>
__global__ void __launch_bounds__(TW, min_ctas2d<T>()) halfstep2d(const Step2D a) {
    constexpr int NV = nvars(SYS), NQ = nq(P), NQ1 = nq(P - 1);
    constexpr int NF = record_fields<SYS, P>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);  // [2][NF][TW]

    const int t = threadIdx.x;
    const int off = a.parity ? -1 : 0;
    const int i0 = blockIdx.x * (TW - 1);
    const int j0 = blockIdx.y * a.rows_per_cta;
    const int rows = min(a.rows_per_cta, a.ny_new - j0);

    const double dt = step_dt2d(a);
    const T lamx = (T)(dt * a.inv_dx), lamy = (T)(dt * a.inv_dy);
    const T idx = (T)a.inv_dx, idy = (T)a.inv_dy;

    const T* in = static_cast<const T*>(a.in);
    T* out = static_cast<T*>(a.out);
    const int pc = parent_index(i0 + t + off, a.nx_old, a.bc);
    T rate_max = 0;
    unsigned err = 0;

    for (int s = 0; s <= rows; ++s) {
        {
            const int pr = parent_index(j0 + off + s, a.ny_old, a.bc);
            long long cell = (long long)pr * a.pitch + pc;
#ifdef WCC2D_BOUNDS_CHECK
            // opt-in checked build: an out-of-range parent is recorded and cell 0 read instead
            if (pr < 0 || pr >= a.rows_alloc || pc < 0 || pc >= a.pitch) {
                atomicOr(&a.st->err, ERR_BOUNDS);
                cell = 0;
            }
#endif
            T q[NV][NQ];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) q[v][qq] = in[(long long)(v * NQ + qq) * a.plane + cell];
            Parent<SYS, P, T> par;
            parent_terms<SYS, P, T>(q, lamx, lamy, a.law, par);
            T* r = ring + (s & 1) * NF * TW;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
#pragma unroll
                for (int k = 0; k < 4; ++k) r[(v * 4 + k) * TW + t] = par.c[v][k];
#pragma unroll
                for (int qq = 0; qq < NQ1; ++qq) r[(NV * 4 + v * NQ1 + qq) * TW + t] = par.V[v][qq];
            }
        }
        __syncthreads();
        if (s >= 1 && t < TW - 1 && i0 + t < a.nx_new) {
            const RingReader<T, TW, NV, NQ1> rd{ring + ((s - 1) & 1) * NF * TW, ring + (s & 1) * NF * TW, t};
            T D[NV][NQ], ub[NV];
            linear_cell<SYS, P, T>(rd, D, ub);
            if (a.law.limiter) {
                if constexpr (SYS == EULER) {
                    T vv[4][4];
#pragma unroll
                    for (int v = 0; v < 4; ++v)
#pragma unroll
                        for (int r = 0; r < 4; ++r) vv[v][r] = rd.V(r, v, 0);
                    if (!limit_euler<P, T>(D, ub, vv, lamx, lamy, a.law)) err |= ERR_POSITIVITY;
                } else {
                    T vv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) vv[r] = rd.V(r, 0, 0);
                    limit_scalar<P, T>(D[0], ub[0], vv, a.law);
                }
            }
            const long long cell = (long long)(j0 + s - 1) * a.pitch + (i0 + t);
            bool store = true;
#ifdef WCC2D_BOUNDS_CHECK
            if (j0 + s - 1 >= a.rows_alloc || i0 + t >= a.pitch) {  // recorded, not written
                atomicOr(&a.st->err, ERR_BOUNDS);
                store = false;
            }
#endif
            if (store) {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int qq = 0; qq < NQ; ++qq) out[(long long)(v * NQ + qq) * a.plane + cell] = D[v][qq];
            }
            T centre[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) centre[v] = D[v][0];
            const T rate = cfl_rate<SYS, T>(centre, a.law, idx, idy);
            if (rate != rate) {
                err |= (SYS == EULER && ub[0] == ub[0]) ? ERR_POSITIVITY : ERR_NONFINITE;
                rate_max = (T)INFINITY;
            } else {
                rate_max = rate > rate_max ? rate : rate_max;
            }
        }
        __syncthreads();
    }
    finish2d<T, TW>(rate_max, err, dt, a);
}

// CFL rate of a loaded stage into rate_bits[0] (and the error bits).
template <int SYS, class T>
__global__ void __launch_bounds__(256) stage_rate2d(const T* planes, long long pitch, long long plane, int nx, int ny,
                                                    int nq_, Law2D law, double dx, double dy, DevState2D* st) {
    constexpr int NV = nvars(SYS);
    T m = 0;
    unsigned err = 0;
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long cell = (c / nx) * pitch + (c % nx);
        T centre[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) centre[v] = planes[(long long)(v * nq_) * plane + cell];
        const T r = cfl_rate<SYS, T>(centre, law, (T)(1.0 / dx), (T)(1.0 / dy));
        if (r != r) {
            err |= SYS == EULER ? ERR_POSITIVITY : ERR_NONFINITE;
            m = (T)INFINITY;
        } else if (r > m) {
            m = r;
        }
    }
    double r = (double)m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->rate_bits[0], (unsigned long long)__double_as_longlong(r));
        if (err) atomicOr(&st->err, err);
    }
}

// host [row][col][v][q] FP64 (staging) -> planes of T, and back; one thread
// per (cell, value), consecutive threads on consecutive cells of a plane
template <class T>
__global__ void aos_to_planes2d(const double* aos, T* planes, int nx, int ny, int nd, long long pitch,
                                long long plane) {
    const long long n = (long long)nx * ny;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n * nd;
         g += (long long)gridDim.x * blockDim.x) {
        const long long f = g / n, c = g % n;
        planes[f * plane + (c / nx) * pitch + (c % nx)] = (T)aos[c * nd + f];
    }
}

template <class T>
__global__ void planes_to_aos2d(const T* planes, double* aos, int nx, int ny, int nd, long long pitch,
                                long long plane) {
    const long long n = (long long)nx * ny;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n * nd;
         g += (long long)gridDim.x * blockDim.x) {
        const long long f = g / n, c = g % n;
        aos[c * nd + f] = (double)planes[f * plane + (c / nx) * pitch + (c % nx)];
    }
}

// CTA width of the half-step: 64 threads for FP64, 128 for FP32, narrowed
// in steps of one warp until the shared ring fits in the 48 KB a kernel gets
// without the opt-in attribute (Euler at P = 3: 32 for FP64, 96 for FP32).
template <int SYS, int P, class T>
constexpr int strip_width() {
    int tw = sizeof(T) == 8 ? 64 : 128;
    while (tw > 32 && ring_bytes<T, 1>(record_fields<SYS, P>()) * tw > 48 * 1024 - 256) tw -= 32;
    return tw;
}

// Launch one half-step of system SYS at degree P in type T.
template <int SYS, int P, class T>
cudaError_t launch_halfstep2d_t(const Step2D& a, cudaStream_t stream) {
    constexpr int TW = strip_width<SYS, P, T>();
    constexpr size_t smem = ring_bytes<T, TW>(record_fields<SYS, P>());
    static_assert(smem <= 48 * 1024 - 256, "the shared ring and the static shared words must fit without the opt-in attribute");
    const dim3 grid((a.nx_new + TW - 2) / (TW - 1), (a.ny_new + a.rows_per_cta - 1) / a.rows_per_cta);
    halfstep2d<SYS, P, T, TW><<<grid, TW, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int SYS, class T>
cudaError_t launch_halfstep2d_sys(int P, const Step2D& a, cudaStream_t stream) {
    switch (P) {
        case 1: return launch_halfstep2d_t<SYS, 1, T>(a, stream);
        case 2: return launch_halfstep2d_t<SYS, 2, T>(a, stream);
        case 3: return launch_halfstep2d_t<SYS, 3, T>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int SYS>
cudaError_t launch_stage_rate2d_sys(bool fp32, const void* planes, long long pitch, long long plane, int nx, int ny,
                                    int nq_, const Law2D& law, double dx, double dy, DevState2D* st,
                                    cudaStream_t stream) {
    const long long n = (long long)nx * ny;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 8);
    if (fp32)
        stage_rate2d<SYS, float><<<grid, 256, 0, stream>>>(static_cast<const float*>(planes), pitch, plane, nx, ny,
                                                           nq_, law, dx, dy, st);
    else
        stage_rate2d<SYS, double><<<grid, 256, 0, stream>>>(static_cast<const double*>(planes), pitch, plane, nx,
                                                            ny, nq_, law, dx, dy, st);
    return cudaGetLastError();
}

// --------------------------------------------------------- FP32-mixed kernel

// Stage layout of the FP32-mixed path: plane (v, 0) holds the high part of
// the cell average (not the point value), planes (v, q >= 1) the scaled
// derivatives in float, and plane NV * NQ + v the low part of the average.
// A parent record: per variable its four shares of the children's averages
// and its vertex point value at t^{n+1/2}, float-float pairs stored as
// float2 (pair field v * 4 + k for share k, NV * 4 + v for the vertex value),
// then the vertex derivatives q = 1 .. NQ1 - 1 (float, from float offset
// 10 NV of the record).
template <int SYS, int P>
__host__ __device__ constexpr int record_fields_mx() {
    return nvars(SYS) * (10 + nq(P - 1) - 1);
}


template <int SYS, int P>
constexpr int strip_width_mx() {
    int tw = 128;
    while (tw > 32 && ring_bytes<float, 1>(record_fields_mx<SYS, P>()) * tw > 48 * 1024 - 256) tw -= 32;
    return tw;
}

template <int TW, int NV, int NQ1>
struct RingReaderMx {
    const float* lo;
    const float* hi;
    int t;
    __device__ __forceinline__ float get(int r, int f) const {
        return r == 0 ? lo[f * TW + t] : r == 1 ? lo[f * TW + t + 1] : r == 2 ? hi[f * TW + t + 1] : hi[f * TW + t];
    }
    __device__ __forceinline__ ff get2(int r, int pf) const {
        const float2* l2 = reinterpret_cast<const float2*>(lo);
        const float2* h2 = reinterpret_cast<const float2*>(hi);
        const float2 x = r == 0 ? l2[pf * TW + t] : r == 1 ? l2[pf * TW + t + 1] : r == 2 ? h2[pf * TW + t + 1] : h2[pf * TW + t];
        return ff{x.x, x.y};
    }
    __device__ __forceinline__ ff cf(int r, int v) const { return get2(r, v * 4 + r); }
    __device__ __forceinline__ ff v00(int r, int v) const { return get2(r, NV * 4 + v); }
    __device__ __forceinline__ float V(int r, int v, int q) const {
        return q == 0 ? get2(r, NV * 4 + v).hi : get(r, NV * 10 + v * (NQ1 - 1) + q - 1);
    }
};

template <int SYS, int P, int TW>
__global__ void __launch_bounds__(TW, 4) halfstep2d_mx(const Step2D a) {
    constexpr int NV = nvars(SYS), NQ = nq(P), NQ1 = nq(P - 1);
    constexpr int NF = record_fields_mx<SYS, P>();
    static_assert((NF * TW) % 2 == 0, "the second row buffer of the ring must start on an 8-byte boundary");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);  // [2][NF][TW]

    const int t = threadIdx.x;
    const int off = a.parity ? -1 : 0;
    const int i0 = blockIdx.x * (TW - 1);
    const int j0 = blockIdx.y * a.rows_per_cta;
    const int rows = min(a.rows_per_cta, a.ny_new - j0);

    const double dt = step_dt2d(a);
    // lam rounded to float in every term, the leading flux terms included:
    // the half-step is one of size fl(lam) dx, the same in all its Taylor
    // terms (a float-float lam for the leading terms alone was measured to
    // move the fine-mesh errors away from FP64's, not towards them)
    const float lamx = (float)(dt * a.inv_dx), lamy = (float)(dt * a.inv_dy);
    const float hx = 0.5f * lamx, hy = 0.5f * lamy;
    const float idx = (float)a.inv_dx, idy = (float)a.inv_dy;

    const float* in = static_cast<const float*>(a.in);
    float* out = static_cast<float*>(a.out);
    const int pc = parent_index(i0 + t + off, a.nx_old, a.bc);
    float rate_max = 0.f;
    unsigned err = 0;

    for (int s = 0; s <= rows; ++s) {
        {
            const int pr = parent_index(j0 + off + s, a.ny_old, a.bc);
            const long long cell = (long long)pr * a.pitch + pc;
            float q[NV][NQ];
            ff ub[NV], u00[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                ub[v] = ff{in[(long long)(v * NQ) * a.plane + cell], in[(long long)(NV * NQ + v) * a.plane + cell]};
                q[v][0] = 0.f;
#pragma unroll
                for (int qq = 1; qq < NQ; ++qq) q[v][qq] = in[(long long)(v * NQ + qq) * a.plane + cell];
                u00[v] = wcc::ff_add(ub[v], -even_correction<P>(q[v]));
                q[v][0] = u00[v].hi;
            }
            Parent<SYS, P, float, true> par;
            parent_terms<SYS, P, float, true>(q, lamx, lamy, a.law, par);
            ff F[NV], G[NV];
            lead_flux_ff<SYS>(u00, a.law, F, G);
            float* r = ring + (s & 1) * NF * TW;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                // quarter averages: ubar/4 +- ox +- oy +- oxy with the signs of
                // RU, LU, LD, RD (vertex roles 1..4), plus the edge fluxes
                // hx f_U = tx, hx f_D = bx, hy g_R = ry, hy g_L = ly:
                //   c0 = q4 + ox + oy + oxy + tx + ry,  c1 = q4 - ox + oy - oxy - tx + ly,
                //   c2 = q4 - ox - oy + oxy - bx - ly,  c3 = q4 + ox - oy - oxy + bx - ry.
                // The O(1) parts (q4 and the leading flux terms hx f(u_00),
                // hy g(u_00)) are added exactly, the float parts (the odd
                // terms and the flux corrections) join the low parts.  c3 is
                // taken as ubar - c0 - c1 - c2, so the parent's shares add up
                // to its ubar to float-float rounding.
                const float ox = 0.25f * par.odd[v][0], oy = 0.25f * par.odd[v][1], oxy = 0.25f * par.odd[v][2];
                const float sxy = ox + oy, dxy = ox - oy;
                const float q4h = 0.25f * ub[v].hi, q4l = 0.25f * ub[v].lo;
                const ff hF = ffm_lazy(F[v], hx), hG = ffm_lazy(G[v], hy);
                const float tl = fmaf(hx, par.fl[v][0], hF.lo), bl = fmaf(hx, par.fl[v][1], hF.lo);
                const float rl = fmaf(hy, par.fl[v][2], hG.lo), ll = fmaf(hy, par.fl[v][3], hG.lo);
                ff c[4];
                c[0] = ff_sum4(q4h, hF.hi, hG.hi, sxy + oxy, q4l + (tl + rl));
                c[1] = ff_sum4(q4h, -hF.hi, hG.hi, -(dxy + oxy), q4l + (ll - tl));
                c[2] = ff_sum4(q4h, -hF.hi, -hG.hi, oxy - sxy, q4l - (bl + ll));
                c[3] = ff_rest3(ub[v], c[0], c[1], c[2]);
                float2* r2 = reinterpret_cast<float2*>(r);
#pragma unroll
                for (int k = 0; k < 4; ++k) r2[(v * 4 + k) * TW + t] = make_float2(c[k].hi, c[k].lo);
                const ff v00 = ff_add_u(u00[v], par.V[v][0]);  // read as a pair only
                r2[(NV * 4 + v) * TW + t] = make_float2(v00.hi, v00.lo);
#pragma unroll
                for (int qq = 1; qq < NQ1; ++qq) r[(NV * 10 + v * (NQ1 - 1) + qq - 1) * TW + t] = par.V[v][qq];
            }
        }
        __syncthreads();
        if (s >= 1 && t < TW - 1 && i0 + t < a.nx_new) {
            const RingReaderMx<TW, NV, NQ1> rd{ring + ((s - 1) & 1) * NF * TW, ring + (s & 1) * NF * TW, t};
            float D[NV][NQ];
            ff ub[NV];
            linear_cell_mx<SYS, P>(rd, D, ub);
            if (a.law.limiter) {
                // deviation form: the point value and the vertex values less
                // the average, taken in float-float and rounded, so that the
                // limiter's slopes and residuals near smooth extrema are not
                // float cancellations of O(1) values; the limited point value
                // comes back as a deviation
                if constexpr (SYS == EULER) {
                    float vv[4][4], ubf[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        ubf[v] = ub[v].hi;
                        D[v][0] = -even_correction<P>(D[v]);
#pragma unroll
                        for (int k = 0; k < 4; ++k) vv[v][k] = wcc::ff_sub(rd.v00(k, v), ub[v]).hi;
                    }
                    if (!limit_euler<P, float, true>(D, ubf, vv, lamx, lamy, a.law)) err |= ERR_POSITIVITY;
#pragma unroll
                    for (int v = 0; v < 4; ++v) D[v][0] += ubf[v];
                } else {
                    float vv[4];
                    D[0][0] = -even_correction<P>(D[0]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) vv[k] = wcc::ff_sub(rd.v00(k, 0), ub[0]).hi;
                    limit_scalar<P, float>(D[0], 0.f, vv, a.law);
                    D[0][0] += ub[0].hi;
                }
            }
            // the limiter keeps the cell average (every candidate has mean ubar)
            const long long cell = (long long)(j0 + s - 1) * a.pitch + (i0 + t);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                out[(long long)(v * NQ) * a.plane + cell] = ub[v].hi;
                out[(long long)(NV * NQ + v) * a.plane + cell] = ub[v].lo;
#pragma unroll
                for (int qq = 1; qq < NQ; ++qq) out[(long long)(v * NQ + qq) * a.plane + cell] = D[v][qq];
            }
            float centre[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) centre[v] = D[v][0];
            const float rate = cfl_rate<SYS, float>(centre, a.law, idx, idy);
            if (rate != rate) {
                err |= (SYS == EULER && ub[0].hi == ub[0].hi) ? ERR_POSITIVITY : ERR_NONFINITE;
                rate_max = INFINITY;
            } else {
                rate_max = rate > rate_max ? rate : rate_max;
            }
        }
        __syncthreads();
    }
    finish2d<float, TW>(rate_max, err, dt, a);
}

// host [row][col][v][q] FP64 point values and derivatives <-> FP32-mixed
// planes; one thread per cell (set-up and read-back only)
template <int P>
__global__ void aos_to_planes2d_mx(const double* aos, float* planes, int nx, int ny, int nv, long long pitch,
                                   long long plane) {
    constexpr int NQ = nq(P);
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long cell = (c / nx) * pitch + (c % nx);
        for (int v = 0; v < nv; ++v) {
            const double* d = aos + (c * nv + v) * NQ;
            double ub = d[0];
            unroll<P + 1>([&](auto kc) {
                unroll<P + 1 - kc>([&](auto lc) {
                    constexpr int k = kc, l = lc;
                    if constexpr (k + l > 0 && !(k & 1) && !(l & 1))
                        ub += pow2m(k) / factd(k + 1) * pow2m(l) / factd(l + 1) * d[qidx(k, l)];
                });
            });
            const float hi = (float)ub;
            planes[(long long)(v * NQ) * plane + cell] = hi;
            planes[(long long)(nv * NQ + v) * plane + cell] = (float)(ub - (double)hi);
            for (int qq = 1; qq < NQ; ++qq) planes[(long long)(v * NQ + qq) * plane + cell] = (float)d[qq];
        }
    }
}

template <int P>
__global__ void planes_to_aos2d_mx(const float* planes, double* aos, int nx, int ny, int nv, long long pitch,
                                   long long plane) {
    constexpr int NQ = nq(P);
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long cell = (c / nx) * pitch + (c % nx);
        for (int v = 0; v < nv; ++v) {
            double* d = aos + (c * nv + v) * NQ;
            for (int qq = 1; qq < NQ; ++qq) d[qq] = (double)planes[(long long)(v * NQ + qq) * plane + cell];
            double u = (double)planes[(long long)(v * NQ) * plane + cell] + (double)planes[(long long)(nv * NQ + v) * plane + cell];
            unroll<P + 1>([&](auto kc) {
                unroll<P + 1 - kc>([&](auto lc) {
                    constexpr int k = kc, l = lc;
                    if constexpr (k + l > 0 && !(k & 1) && !(l & 1))
                        u -= pow2m(k) / factd(k + 1) * pow2m(l) / factd(l + 1) * d[qidx(k, l)];
                });
            });
            d[0] = u;
        }
    }
}

// CFL rate of a loaded FP32-mixed stage: the point value from the average
template <int SYS, int P>
__global__ void __launch_bounds__(256) stage_rate2d_mx(const float* planes, long long pitch, long long plane, int nx,
                                                       int ny, Law2D law, double dx, double dy, DevState2D* st) {
    constexpr int NV = nvars(SYS), NQ = nq(P);
    float m = 0.f;
    unsigned err = 0;
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long cell = (c / nx) * pitch + (c % nx);
        float centre[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            float d[NQ];
            d[0] = 0.f;
#pragma unroll
            for (int qq = 1; qq < NQ; ++qq) d[qq] = planes[(long long)(v * NQ + qq) * plane + cell];
            const ff ub{planes[(long long)(v * NQ) * plane + cell], planes[(long long)(NV * NQ + v) * plane + cell]};
            centre[v] = wcc::ff_add(ub, -even_correction<P>(d)).hi;
        }
        const float r = cfl_rate<SYS, float>(centre, law, (float)(1.0 / dx), (float)(1.0 / dy));
        if (r != r) {
            err |= SYS == EULER ? ERR_POSITIVITY : ERR_NONFINITE;
            m = INFINITY;
        } else if (r > m) {
            m = r;
        }
    }
    double r = (double)m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->rate_bits[0], (unsigned long long)__double_as_longlong(r));
        if (err) atomicOr(&st->err, err);
    }
}

template <int SYS, int P>
cudaError_t launch_halfstep2d_mx_t(const Step2D& a, cudaStream_t stream) {
    constexpr int TW = strip_width_mx<SYS, P>();
    constexpr size_t smem = ring_bytes<float, TW>(record_fields_mx<SYS, P>());
    static_assert(smem <= 48 * 1024 - 256, "the shared ring and the static shared words must fit without the opt-in attribute");
    const dim3 grid((a.nx_new + TW - 2) / (TW - 1), (a.ny_new + a.rows_per_cta - 1) / a.rows_per_cta);
    halfstep2d_mx<SYS, P, TW><<<grid, TW, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace wcc2d

namespace wcc2d {
// Instantiated in wcc2d_mixed.cu.
cudaError_t launch_halfstep2d_mx(int system, int P, const Step2D& a, cudaStream_t stream);
cudaError_t launch_stage_rate2d_mx(int system, int P, const float* planes, long long pitch, long long plane, int nx,
                                   int ny, const Law2D& law, double dx, double dy, DevState2D* st, cudaStream_t stream);
cudaError_t launch_convert2d_mx(int P, bool to_planes, double* aos, float* planes, int nx, int ny, int nv,
                                long long pitch, long long plane, cudaStream_t stream);
}  // namespace wcc2d

namespace wcc2d {
// Instantiated in wcc2d_scalar.cu, wcc2d_euler_f64.cu, wcc2d_euler_f32.cu.
cudaError_t launch_halfstep2d(int system, int P, bool fp32, const Step2D& a, cudaStream_t stream);
cudaError_t launch_stage_rate2d(int system, bool fp32, const void* planes, long long pitch, long long plane, int nx,
                                int ny, int nq_, const Law2D& law, double dx, double dy, DevState2D* st,
                                cudaStream_t stream);
}  // namespace wcc2d
