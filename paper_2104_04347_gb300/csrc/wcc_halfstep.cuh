// wcc_halfstep.cuh -- the fused half-step kernel (FP64 instantiation) and
// the small auxiliary kernels (stage CFL bound, layout conversion).
//
// One launch advances a whole stage by one staggered half-step
// (Sec. 2.1, Fig. 1).  Each CTA:
//   1. loads kThreads parent cells (coalesced: consecutive threads read
//      consecutive cells of each [var][k] plane), runs the Cauchy-Kovalewski
//      procedure once per parent, and keeps the parent record (two flux /
//      half-average contributions and the vertex Taylor coefficients) in
//      shared memory -- each parent is a vertex of two new cells;
//   2. builds kTile new cells from neighbouring records: finite-volume cell
//      average, central-difference derivatives, point value, limiter;
//   3. reduces the new stage's largest characteristic speed (warp shuffles,
//      one atomic per CTA); the last CTA to finish publishes the stage bound,
//      advances t and records dt, so the next launch derives its dt on the
//      device without a host round trip.
#pragma once

#include "wcc_scheme.cuh"

namespace wcc {

__device__ __forceinline__ long long parent_index(long long p, long long n, int bc) {
    if (bc == BC_PERIODIC) {
        if (p < 0) p += n;
        if (p >= n) p -= n;
        if (p < 0 || p >= n) p = ((p % n) + n) % n;  // tail CTAs reach past one period
        return p;
    }
    // transmissive: ghost staggered cells copy the adjacent cell
    return p < 0 ? 0 : (p >= n ? n - 1 : p);
}

template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Bookkeeping of a solver state after the last CTA of a half-step finished:
// publish the new stage's bound, clear the slots the next launches
// accumulate into, record dt, advance t and prepare the next CFL step.
// FP32 kernels (f32) accumulate the bound in amax_f32.
__device__ __forceinline__ void finalize_state(DevState* st, bool f32, double dt, double* hist, long long hist_cap,
                                               int parity, int cfl_mode, double cfl, double dx) {
    if (f32) {
        const float fm = __uint_as_float(st->amax_f32[parity ^ 1]);
        st->amax_bits[parity ^ 1] = (unsigned long long)__double_as_longlong((double)fm);
        st->amax_f32[parity] = 0u;
    }
    // Every CTA of this launch has read amax_bits[parity]; clear it for the
    // launch after next, which accumulates into it.
    st->amax_bits[parity] = 0ull;
    const long long k = st->step;
    if (k < hist_cap) hist[k] = dt;
    st->step = k + 1;
    st->t = st->t + dt;
    st->blocks_done = 0u;
    if (not_finite(dt)) st->err |= ERR_NONFINITE;
    if (cfl_mode) {
        const double amax = __longlong_as_double((long long)st->amax_bits[parity ^ 1]);
        const double ndt = cfl * dx / amax;
        const double nlam = ndt / dx;
        st->next_dt = ndt;
        st->next_lam = nlam;
        split_to_floats(nlam, st->next_lam_hi, st->next_lam_lo);
        st->next_cfl = cfl;
    } else {
        st->next_cfl = 0.0;
    }
    __threadfence();
}

// Block-wide max of the speed (in the kernel's compute type T), one atomic
// per CTA into st, then count the CTA as done; the CTA that completes the
// `ctas` of this state does its bookkeeping.  Synchronises the block.
template <class T, int NT = kThreads>
__device__ __forceinline__ void reduce_and_finish(T speed, unsigned err, double dt, DevState* st, long long ctas,
                                                  double* hist, long long hist_cap, int parity, int cfl_mode,
                                                  double cfl, double dx) {
    // One block barrier: the warps' maxima and error bits meet in shared
    // memory, thread 0 combines them, posts them and counts the CTA; the CTA
    // that counts last finishes the launch's bookkeeping.  The barrier also
    // guarantees that every warp is done with the tile's shared records.
    __shared__ T s_max[NT / 32];
    __shared__ unsigned s_err[NT / 32];
    // NaN must win the max: map it to +Inf and flag it
    if (speed != speed) {
        speed = (T)INFINITY;
        err |= ERR_NONFINITE;
    }
    speed = warp_max<T>(speed);
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
        s_max[threadIdx.x >> 5] = speed;
        s_err[threadIdx.x >> 5] = err;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = s_max[0];
        unsigned e = s_err[0];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w) {
            m = fmax(m, s_max[w]);
            e |= s_err[w];
        }
        if constexpr (sizeof(T) == 8) {
            if (m > 0.0) atomicMax(&st->amax_bits[parity ^ 1], (unsigned long long)__double_as_longlong(m));
        } else {
            if (m > 0.f) atomicMax(&st->amax_f32[parity ^ 1], __float_as_uint(m));
        }
        if (e) atomicOr(&st->err, e);
        __threadfence();
        const unsigned done = atomicAdd(&st->blocks_done, 1u);
        if (done == (unsigned)(ctas - 1)) {
            __threadfence();
            finalize_state(st, sizeof(T) == 4, dt, hist, hist_cap, parity, cfl_mode, cfl, dx);
        }
    }
}
template <class T, int NT = kThreads>
__device__ __forceinline__ void finish_halfstep(T speed, unsigned err, double dt, const StepArgs& args) {
    reduce_and_finish<T, NT>(speed, err, dt, args.st, (long long)gridDim.x, args.hist, args.hist_cap, args.parity,
                             args.cfl_mode, args.cfl, args.dx);
}

template <int SYS, int P>
__global__ void __launch_bounds__(kThreads) halfstep_fp64(const StepArgs args) {
    constexpr int NV = nvars(SYS);
    constexpr int K = P + 1;
    constexpr int NREC = NV * (P + 3);
    __shared__ double rec[NREC][kThreads];

    const int t = threadIdx.x;
    const long long first_new = (long long)blockIdx.x * kTile;

    const StepSize z = step_size(args);
    const double dt = z.dt;
    const double lam = z.lam;

    // ---- phase 1: parent record of parent slot t
    {
        const long long p = parent_index(first_new + t - (args.parity ? 1 : 0), args.n_old, args.bc);
        double c[NV][K];
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            sfor<0, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                c[v][k] = __ldg(args.in64 + (long long)(v * K + k) * args.pitch + p);
            });
        });
        ParentRecord<SYS, P, double> r;
        parent_record<SYS, P, double>(c, lam, args, r);
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            rec[v][t] = r.A[v];
            rec[NV + v][t] = r.B[v];
            sfor<0, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                rec[2 * NV + v * K + k][t] = r.vtx[v][k];
            });
        });
    }
    __syncthreads();

    // ---- phase 2: new cell t from parent slots t (left) and t + 1 (right)
    const long long i = first_new + t;
    double speed = 0.0;
    unsigned err = 0u;
    if (t < kTile && i < args.n_new) {
        double e[NV][K], ubar[NV], vl[NV], vr[NV];
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            double vL[K], vR[K];
            sfor<0, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                vL[k] = rec[2 * NV + v * K + k][t];
                vR[k] = rec[2 * NV + v * K + k][t + 1];
            });
            ubar[v] = rec[v][t] + rec[NV + v][t + 1];
            vl[v] = vL[0];
            vr[v] = vR[0];
            derivatives_and_point_value<P, double>(ubar[v], vL, vR, e[v]);
        });

        if (args.limiter) {
            if constexpr (NV == 1) {
                limit_scalar<P, double>(e[0], ubar[0], vl[0], vr[0], args);
            } else {
                // Sec. 4: limit characteristic variables L(ubar) U, map back with R(ubar).
                EulerChar<double> E;
                if (!euler_char<double>(ubar, args.gamma, E)) err |= ERR_POSITIVITY;
                double ce[3][K], cub[3], cvl[3], cvr[3];
                E.left(ubar[0], ubar[1], ubar[2], cub);
                E.left(vl[0], vl[1], vl[2], cvl);
                E.left(vr[0], vr[1], vr[2], cvr);
                sfor<0, K>([&](auto Ki) {
                    constexpr int k = decltype(Ki)::value;
                    double w[3];
                    E.left(e[0][k], e[1][k], e[2][k], w);
                    ce[0][k] = w[0];
                    ce[1][k] = w[1];
                    ce[2][k] = w[2];
                });
                sfor<0, 3>([&](auto Ii) {
                    constexpr int r = decltype(Ii)::value;
                    limit_scalar<P, double>(ce[r], cub[r], cvl[r], cvr[r], args);
                });
                sfor<0, K>([&](auto Ki) {
                    constexpr int k = decltype(Ki)::value;
                    E.right(ce[0][k], ce[1][k], ce[2][k], e[0][k], e[1][k], e[2][k]);
                });
            }
        }

        bool bad = false;
        sfor<0, NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            sfor<0, K>([&](auto Ki) {
                constexpr int k = decltype(Ki)::value;
                bad |= not_finite(e[v][k]);
                __stcs(args.out64 + (long long)(v * K + k) * args.pitch + i, e[v][k]);
            });
        });
        if (bad) err |= ERR_NONFINITE;
        double u0[NV];
        sfor<0, NV>([&](auto V) { u0[decltype(V)::value] = e[decltype(V)::value][0]; });
        speed = wave_speed<SYS, double>(u0, args, err);
    }
    finish_halfstep<double>(speed, err, dt, args);
}

// Largest characteristic speed of a stage (used once after loading data).
template <int SYS>
__global__ void __launch_bounds__(256) stage_speed(const double* u0planes, long long var_stride, long long n,
                                                    StepArgs args, int slot) {
    constexpr int NV = nvars(SYS);
    double m = 0.0;
    unsigned err = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double u0[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u0[v] = u0planes[v * var_stride + i];
        double s = wave_speed<SYS, double>(u0, args, err);
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
