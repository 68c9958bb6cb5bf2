// wcc_api.cu -- the C ABI of include/wcc.h: solver handle, device memory,
// layout conversion, time marching with device-side dt and CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/wcc.h"
#include "wcc_launch.h"
#include "wcc_convert.cuh"
#include "wcc_mixed2.cuh"
#include "wcc_ff.cuh"
#include "wcc_scheme.cuh"
#include "wcc_trace.h"

using namespace wcc;

namespace {

thread_local std::string g_create_error;

// ------------------------------------------------ layout conversion kernels

// Host layout [cell][var][k] of paper-scaled derivatives u_kx  <->  device
// planes of Taylor coefficients e_k = u_kx / k!.  Each CTA converts a tile of
// kConvCells cells through shared memory: the host-layout side of the tile is
// one contiguous run of doubles and the plane side one run per plane, so both
// global sides are coalesced.
// 1/k! and k! for k = 0..6, rounded once to double (the layout conversions
// multiply by these instead of dividing: FP64 division is slow on this GPU).
__device__ __forceinline__ double inv_fact_k(int k) {
    const double t[7] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0};
    return t[k];
}
__device__ __forceinline__ double fact_k(int k) {
    const double t[7] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0};
    return t[k];
}

constexpr int kConvCells = 128;                 // cells per tile
constexpr int kConvThreads = 256;
constexpr int kConvMaxElems = kConvCells * 3 * 7;  // nv <= 3, K <= 7

// Copies cells [c0, c0 + m) of the host-layout array to / from smem (as
// doubles, or as their bit patterns for the FP32-mixed conversions).
template <class T>
__device__ __forceinline__ void tile_load(const T* __restrict__ aos, long long c0, int m, int row, T* sm) {
    const T* src = aos + c0 * row;
    for (int i = threadIdx.x; i < m * row; i += kConvThreads) sm[i] = src[i];
}
template <class T>
__device__ __forceinline__ void tile_store(T* __restrict__ aos, long long c0, int m, int row, const T* sm) {
    T* dst = aos + c0 * row;
    for (int i = threadIdx.x; i < m * row; i += kConvThreads) dst[i] = sm[i];
}

__global__ void __launch_bounds__(kConvThreads) aos_to_planes_fp64(const double* __restrict__ aos, long long n,
                                                                   int nv, int K, long long pitch,
                                                                   double* __restrict__ planes) {
    __shared__ double sm[kConvMaxElems];
    const int row = nv * K;
    for (long long c0 = (long long)blockIdx.x * kConvCells; c0 < n; c0 += (long long)gridDim.x * kConvCells) {
        const int m = (int)min((long long)kConvCells, n - c0);
        tile_load(aos, c0, m, row, sm);
        __syncthreads();
        // element (plane q = v K + k, cell c): consecutive threads, consecutive cells
        for (int i = threadIdx.x; i < kConvCells * row; i += kConvThreads) {
            const int c = i % kConvCells, q = i / kConvCells;
            if (c < m) planes[(long long)q * pitch + c0 + c] = sm[c * row + q] * inv_fact_k(q % K);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kConvThreads) planes_to_aos_fp64(const double* __restrict__ planes, long long n,
                                                                   int nv, int K, long long pitch,
                                                                   double* __restrict__ aos) {
    __shared__ double sm[kConvMaxElems];
    const int row = nv * K;
    for (long long c0 = (long long)blockIdx.x * kConvCells; c0 < n; c0 += (long long)gridDim.x * kConvCells) {
        const int m = (int)min((long long)kConvCells, n - c0);
        for (int i = threadIdx.x; i < kConvCells * row; i += kConvThreads) {
            const int c = i % kConvCells, q = i / kConvCells;
            if (c < m) sm[c * row + q] = planes[(long long)q * pitch + c0 + c] * fact_k(q % K);
        }
        __syncthreads();
        tile_store(aos, c0, m, row, sm);
        __syncthreads();
    }
}

// FP32-mixed / FP32 host layout from the planes (the set-up direction is
// load_stage_mixed, which also takes the stage's CFL bound).
template <int K>
__global__ void __launch_bounds__(kConvThreads) planes_to_aos_mixed(const float* __restrict__ planes, long long n,
                                                                    int nv, long long pitch,
                                                                    double* __restrict__ aos) {
    __shared__ unsigned long long sm[kConvMaxElems];  // DOFs as bit patterns
    constexpr int NP = K + 1;
    const int row = nv * K;
    for (long long c0 = (long long)blockIdx.x * kConvCells; c0 < n; c0 += (long long)gridDim.x * kConvCells) {
        const int m = (int)min((long long)kConvCells, n - c0);
        for (int i = threadIdx.x; i < kConvCells * nv; i += kConvThreads) {
            const int c = i % kConvCells, v = i / kConvCells;
            if (c >= m) continue;
            const float* pl = planes + (long long)(v * NP) * pitch + c0 + c;
            float e[K];
#pragma unroll
            for (int k = 1; k < K; ++k) e[k] = pl[(long long)(k + 1) * pitch];
            mixed_to_host<K>(ff{pl[0], pl[pitch]}, e, sm + c * row + v * K);
        }
        __syncthreads();
        tile_store(reinterpret_cast<unsigned long long*>(aos), c0, m, row, sm);
        __syncthreads();
    }
}

// Launch helper: K = P + 1 as a template argument.
cudaError_t launch_planes_to_aos_mixed(int K, unsigned grid, cudaStream_t s, const float* planes, long long n, int nv,
                                       long long pitch, double* aos) {
    switch (K) {
        case 2: planes_to_aos_mixed<2><<<grid, kConvThreads, 0, s>>>(planes, n, nv, pitch, aos); break;
        case 3: planes_to_aos_mixed<3><<<grid, kConvThreads, 0, s>>>(planes, n, nv, pitch, aos); break;
        case 4: planes_to_aos_mixed<4><<<grid, kConvThreads, 0, s>>>(planes, n, nv, pitch, aos); break;
        case 5: planes_to_aos_mixed<5><<<grid, kConvThreads, 0, s>>>(planes, n, nv, pitch, aos); break;
        case 6: planes_to_aos_mixed<6><<<grid, kConvThreads, 0, s>>>(planes, n, nv, pitch, aos); break;
        case 7: planes_to_aos_mixed<7><<<grid, kConvThreads, 0, s>>>(planes, n, nv, pitch, aos); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Tiles of the conversion kernels: one per kConvCells cells, at most 8 CTAs
// per SM of a 152-SM GPU (the kernels stride over the rest).
unsigned conv_grid(long long n) {
    long long b = (n + kConvCells - 1) / kConvCells;
    if (b > 152 * 8) b = 152 * 8;
    return (unsigned)(b < 1 ? 1 : b);
}


}  // namespace

struct wcc_ctx {
    int system = 0, P = 0, nv = 1, K = 2, bc = 0;
    long long N = 0;
    double xl = 0, xr = 1, dx = 1;
    wcc_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;

    long long pitch = 0;
    double* s64[2] = {nullptr, nullptr};  // FP64 stages
    float* s32[2] = {nullptr, nullptr};   // FP32-mixed stages
    double* staging = nullptr;  // host-layout FP64 staging buffer
    DevState* st = nullptr;
    double* hist = nullptr;
    long long hist_cap = 0;
    long long bytes = 0;

    int cur = 0;          // buffer holding the current stage
    int parity = 0;       // stage parity of the current stage
    long long steps = 0;  // half-steps since wcc_set_initial
    bool initialised = false;

    cudaGraphExec_t gexec = nullptr;
    int g_cur = -1, g_parity = -1, g_chunk = 0;
    double g_cfl = 0.0;
    // two half-steps per launch (tb_depth = 2)
    cudaGraphExec_t gexec_tb = nullptr;
    int gt_cur = -1, gt_parity = -1, gt_pairs = 0;
    double gt_cfl = 0.0;
    double tb_limit = 0.0;  // wcc_stability_limit(P)
    long long tb_pairs = 0, tb_fallbacks = 0;

    long long launches = 0;
    std::string err;
};

namespace {

int fail(wcc_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg; else g_create_error = msg;
    return code;
}

int cuda_fail(wcc_ctx* h, cudaError_t e, const char* what) {
    return fail(h, WCC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define WCC_CHECK(h, call)                                              \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);        \
    } while (0)

long long stage_cells(const wcc_ctx* h, int parity) {
    if (h->bc == WCC_BC_PERIODIC) return h->N;
    return parity == 0 ? h->N + 1 : h->N;
}

long long next_cells(const wcc_ctx* h, int parity) { return stage_cells(h, parity ^ 1); }

cudaError_t launch_pair_kernel(wcc_ctx* h, const StepArgs& a) {
    switch (h->system) {
        case WCC_ADVECTION: return launch_halfstep_pair<ADVECTION>(h->P, h->opt.precision, a, h->stream);
        case WCC_BURGERS: return launch_halfstep_pair<BURGERS>(h->P, h->opt.precision, a, h->stream);
        default: return launch_halfstep_pair<EULER>(h->P, h->opt.precision, a, h->stream);
    }
}

cudaError_t launch_step_kernel(wcc_ctx* h, const StepArgs& a) {
    switch (h->system) {
        case WCC_ADVECTION: return launch_halfstep<ADVECTION>(h->P, h->opt.precision, a, h->stream);
        case WCC_BURGERS: return launch_halfstep<BURGERS>(h->P, h->opt.precision, a, h->stream);
        default: return launch_halfstep<EULER>(h->P, h->opt.precision, a, h->stream);
    }
}

StepArgs make_args(wcc_ctx* h, int cur, int parity, double cfl, double dt_fixed) {
    StepArgs a{};
    a.in64 = h->s64[cur];
    a.out64 = h->s64[cur ^ 1];
    a.in32 = h->s32[cur];
    a.out32 = h->s32[cur ^ 1];
    a.pitch = h->pitch;
    a.n_old = stage_cells(h, parity);
    a.n_new = next_cells(h, parity);
    a.parity = parity;
    a.bc = h->bc;
    a.limiter = h->opt.limiter;
    a.alpha_is_two = (h->opt.alpha == 2.0);
    a.dx = h->dx;
    a.cfl = cfl;
    a.cfl_mode = cfl > 0.0 ? 1 : 0;
    a.cfl_bits = (unsigned long long)__double_as_longlong_host(cfl);
    a.dt_fixed = dt_fixed;
    a.lam_fixed = dt_fixed / h->dx;
    split_double(a.lam_fixed, a.lam_fixed_hi, a.lam_fixed_lo);
    a.adv = h->opt.adv_speed;
    a.gamma = h->opt.gamma;
    a.alpha = h->opt.alpha;
    a.eps = h->opt.eps;
    a.st = h->st;
    a.hist = h->hist;
    a.hist_cap = h->hist_cap;
    a.gamma_f = (float)h->opt.gamma;
    split_double(h->opt.gamma - 1.0, a.g1_hi, a.g1_lo);
    split_double(h->opt.adv_speed, a.adv_hi, a.adv_lo);
    a.eps_f = (float)h->opt.eps;
    a.alpha_f = (float)h->opt.alpha;
    a.n_mid = stage_cells(h, parity ^ 1);
    a.tb_nu_max = std::min(cfl * (1.0 + h->opt.tb_cfl_growth), h->tb_limit);
    a.tiles_per_cta = (h->opt.precision == WCC_FP64 || h->opt.cells_per_block == 0)
                          ? 0 : h->opt.cells_per_block / kTileMixed;
    return a;
}

int read_state(wcc_ctx* h, DevState* out) {
    WCC_CHECK(h, cudaStreamSynchronize(h->stream));
    WCC_CHECK(h, cudaMemcpy(out, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    // the more specific cause first: a negative density also makes c NaN
    if (out->err & ERR_POSITIVITY)
        return fail(h, WCC_E_POSITIVITY, "non-positive density or pressure at a cell centre");
    if (out->err & ERR_NONFINITE) return fail(h, WCC_E_NONFINITE, "a DOF or the CFL bound became NaN/Inf");
    return WCC_OK;
}

int ensure_history(wcc_ctx* h, long long need) {
    if (need <= h->hist_cap) return WCC_OK;
    long long cap = h->hist_cap > 0 ? h->hist_cap : 1024;
    while (cap < need) cap *= 2;
    double* nh = nullptr;
    WCC_CHECK(h, cudaStreamSynchronize(h->stream));
    cudaError_t e = cudaMalloc(&nh, cap * sizeof(double));
    if (e != cudaSuccess) return fail(h, WCC_E_NOMEM, "cudaMalloc of the dt history failed");
    if (h->hist) {
        WCC_CHECK(h, cudaMemcpy(nh, h->hist, h->hist_cap * sizeof(double), cudaMemcpyDeviceToDevice));
        cudaFree(h->hist);
    }
    h->bytes += (cap - h->hist_cap) * (long long)sizeof(double);
    h->hist = nh;
    h->hist_cap = cap;
    if (h->gexec) {  // captured launches hold the old pointer
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    if (h->gexec_tb) {
        cudaGraphExecDestroy(h->gexec_tb);
        h->gexec_tb = nullptr;
    }
    return WCC_OK;
}

int enqueue_one(wcc_ctx* h, double cfl, double dt_fixed) {
    StepArgs a = make_args(h, h->cur, h->parity, cfl, dt_fixed);
    cudaError_t e = launch_step_kernel(h, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "half-step launch");
    h->launches += 1;
    h->cur ^= 1;
    h->parity ^= 1;
    h->steps += 1;
    return WCC_OK;
}

// Capture `chunk` (even) CFL half-steps starting from the current buffer and
// parity into one graph; after it the buffer and parity are unchanged.
int build_graph(wcc_ctx* h, int chunk, double cfl) {
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    WCC_CHECK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int cur = h->cur, parity = h->parity;
    for (int s = 0; s < chunk; ++s) {
        StepArgs a = make_args(h, cur, parity, cfl, 0.0);
        cudaError_t e = launch_step_kernel(h, a);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            return cuda_fail(h, e, "half-step launch during capture");
        }
        cur ^= 1;
        parity ^= 1;
    }
    WCC_CHECK(h, cudaStreamEndCapture(h->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->gexec = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    h->g_cur = h->cur;
    h->g_parity = h->parity;
    h->g_cfl = cfl;
    h->g_chunk = chunk;
    return WCC_OK;
}

// Two half-steps in one launch from the current buffer (parity unchanged).
// Arguments of a two-half-step launch: the final stage has the parity, and
// so the cell count, of the input stage.
StepArgs make_pair_args(wcc_ctx* h, int cur, double cfl) {
    StepArgs a = make_args(h, cur, h->parity, cfl, 0.0);
    a.n_new = a.n_old;
    return a;
}

int enqueue_pair(wcc_ctx* h, double cfl) {
    StepArgs a = make_pair_args(h, h->cur, cfl);
    cudaError_t e = launch_pair_kernel(h, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "two-half-step launch");
    h->launches += 1;
    h->cur ^= 1;
    h->steps += 2;
    return WCC_OK;
}

// Capture `pairs` (even) two-half-step launches from the current buffer and
// parity into one graph; after it the buffer and parity are unchanged.
int build_graph_pairs(wcc_ctx* h, int pairs, double cfl) {
    if (h->gexec_tb) {
        cudaGraphExecDestroy(h->gexec_tb);
        h->gexec_tb = nullptr;
    }
    cudaGraph_t g = nullptr;
    WCC_CHECK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int cur = h->cur;
    for (int s = 0; s < pairs; ++s) {
        StepArgs a = make_pair_args(h, cur, cfl);
        cudaError_t e = launch_pair_kernel(h, a);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            return cuda_fail(h, e, "two-half-step launch during capture");
        }
        cur ^= 1;
    }
    WCC_CHECK(h, cudaStreamEndCapture(h->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&h->gexec_tb, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->gexec_tb = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    h->gt_cur = h->cur;
    h->gt_parity = h->parity;
    h->gt_cfl = cfl;
    h->gt_pairs = pairs;
    return WCC_OK;
}

void release(wcc_ctx* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gexec_tb) cudaGraphExecDestroy(h->gexec_tb);
    for (int i = 0; i < 2; ++i) {
        if (h->s64[i]) cudaFree(h->s64[i]);
        if (h->s32[i]) cudaFree(h->s32[i]);
    }
    if (h->staging) cudaFree(h->staging);
    if (h->st) cudaFree(h->st);
    if (h->hist) cudaFree(h->hist);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}


// nsteps single CFL half-steps: graphs of graph_chunk, then direct launches.
int step_single(wcc_ctx* h, long long nsteps, double cfl) {
    int rc;
    long long left = nsteps;
    const int chunk = h->opt.graph_chunk;
    if (chunk >= 2 && h->stream != nullptr && left >= chunk) {
        if (!h->gexec || h->g_cur != h->cur || h->g_parity != h->parity || h->g_cfl != cfl ||
            h->g_chunk != chunk) {
            rc = build_graph(h, chunk, cfl);
            if (rc != WCC_OK) return rc;
        }
        while (left >= chunk) {
            WCC_CHECK(h, cudaGraphLaunch(h->gexec, h->stream));
            h->launches += chunk;
            h->steps += chunk;
            left -= chunk;
        }
    }
    for (; left > 0; --left) {
        rc = enqueue_one(h, cfl, 0.0);
        if (rc != WCC_OK) return rc;
    }
    return WCC_OK;
}

// nsteps CFL half-steps as two-half-step launches (an odd last one single),
// checked after the launches: a pair refused by its CFL check (ERR_CFL; it
// and the launches queued after it changed nothing) is re-done as two single
// half-steps from the last stage reached, and the pairs resume.
int step_pairs(wcc_ctx* h, long long nsteps, double cfl) {
    long long pairs = nsteps / 2;
    const int graph_pairs = (h->opt.graph_chunk / 2) & ~1;  // even: the graph keeps cur
    while (pairs > 0) {
        const int cur0 = h->cur;
        const long long steps0 = h->steps;
        long long left = pairs;
        int rc;
        if (graph_pairs >= 2 && h->stream != nullptr && left >= graph_pairs) {
            if (!h->gexec_tb || h->gt_cur != h->cur || h->gt_parity != h->parity || h->gt_cfl != cfl ||
                h->gt_pairs != graph_pairs) {
                if ((rc = build_graph_pairs(h, graph_pairs, cfl)) != WCC_OK) return rc;
            }
            while (left >= graph_pairs) {
                WCC_CHECK(h, cudaGraphLaunch(h->gexec_tb, h->stream));
                h->launches += graph_pairs;
                h->steps += 2 * graph_pairs;
                left -= graph_pairs;
            }
        }
        for (; left > 0; --left)
            if ((rc = enqueue_pair(h, cfl)) != WCC_OK) return rc;
        DevState st;
        if ((rc = read_state(h, &st)) != WCC_OK) return rc;
        if (!(st.err & ERR_CFL)) {
            h->tb_pairs += pairs;
            break;
        }
        // refused: the device state is at the last stage reached
        const long long done_pairs = (st.step - steps0) / 2;
        h->tb_pairs += done_pairs;
        h->tb_fallbacks += 1;
        h->cur = cur0 ^ (int)(done_pairs & 1);
        h->steps = st.step;
        const unsigned e = st.err & ~ERR_CFL;
        WCC_CHECK(h, cudaMemcpy(&h->st->err, &e, sizeof e, cudaMemcpyHostToDevice));
        for (int k = 0; k < 2; ++k)
            if ((rc = enqueue_one(h, cfl, 0.0)) != WCC_OK) return rc;
        pairs -= done_pairs + 1;
    }
    if (nsteps & 1) return enqueue_one(h, cfl, 0.0);
    return WCC_OK;
}

}  // namespace

extern "C" {

void wcc_default_options(wcc_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = WCC_FP64;
    opt->limiter = 1;
    opt->alpha = 2.0;
    opt->eps = 1e-40;
    opt->gamma = 1.4;
    opt->adv_speed = 1.0;
    opt->graph_chunk = 32;
    opt->tb_depth = 1;
    opt->cuda_stream = nullptr;
    opt->tb_cfl_growth = 0.1;
    opt->cells_per_block = 0;
    opt->reserved = 0;
}

int wcc_create(wcc_handle* out, int system, int64_t N, int P, const double domain[2], int bc,
               const wcc_options* opt) {
    if (!out) return fail(nullptr, WCC_E_INVAL, "out is NULL");
    *out = nullptr;
    if (system < WCC_ADVECTION || system > WCC_EULER) return fail(nullptr, WCC_E_INVAL, "unknown system");
    if (P < 1 || P > 6) return fail(nullptr, WCC_E_INVAL, "P must be in 1..6");
    if (N < 4 || N > (1ll << 31)) return fail(nullptr, WCC_E_INVAL, "N must be in 4..2^31");
    if (!domain || !(domain[1] > domain[0])) return fail(nullptr, WCC_E_INVAL, "domain must satisfy x_L < x_R");
    if (bc != WCC_BC_PERIODIC && bc != WCC_BC_TRANSMISSIVE) return fail(nullptr, WCC_E_INVAL, "unknown bc");
    wcc_options o;
    wcc_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != WCC_FP64 && o.precision != WCC_FP32_MIXED && o.precision != WCC_FP32)
        return fail(nullptr, WCC_E_INVAL, "precision must be WCC_FP64, WCC_FP32_MIXED or WCC_FP32");
    if (!(o.eps >= 0.0) || !(o.alpha > 0.0) || !(o.gamma > 1.0))
        return fail(nullptr, WCC_E_INVAL, "need eps >= 0, alpha > 0, gamma > 1");
    if (o.graph_chunk < 0) return fail(nullptr, WCC_E_INVAL, "graph_chunk must be >= 0");
    if (o.tb_depth == 0) o.tb_depth = 1;
    if (o.tb_depth != 1 && o.tb_depth != 2) return fail(nullptr, WCC_E_INVAL, "tb_depth must be 1 or 2");
    if (o.tb_depth == 2 && o.precision == WCC_FP64)
        return fail(nullptr, WCC_E_INVAL, "tb_depth = 2 needs WCC_FP32_MIXED or WCC_FP32");
    if (!(o.tb_cfl_growth >= -1.0) || !(o.tb_cfl_growth < 1e6))
        return fail(nullptr, WCC_E_INVAL, "tb_cfl_growth must be a number >= -1");
    {
        const int c = o.cells_per_block;
        const bool ok = c == 0 ||
                        (o.precision == WCC_FP64 && c == kTile) ||
                        (o.precision == WCC_FP32_MIXED && (c == kTileMixed || c == 2 * kTileMixed)) ||
                        (o.precision == WCC_FP32 && c == kTileMixed * mixed_default_tiles(P));
        if (!ok) return fail(nullptr, WCC_E_INVAL, "cells_per_block is not a compiled tile size for this precision");
    }
    double tb_limit = 0.0;
    if (o.tb_depth == 2 && wcc_stability_limit(P, &tb_limit) != WCC_OK)
        return fail(nullptr, WCC_E_INVAL, "no stability limit for this P");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(nullptr, WCC_E_CUDA, "no CUDA device available");

    wcc_ctx* h = new (std::nothrow) wcc_ctx();
    if (!h) return fail(nullptr, WCC_E_NOMEM, "host allocation failed");
    h->system = system;
    h->P = P;
    h->nv = (system == WCC_EULER) ? 3 : 1;
    h->K = P + 1;
    h->bc = bc;
    h->N = N;
    h->xl = domain[0];
    h->xr = domain[1];
    h->dx = (domain[1] - domain[0]) / (double)N;
    h->opt = o;
    h->tb_limit = tb_limit;
    if (h->opt.graph_chunk & 1) h->opt.graph_chunk += 1;
    cudaGetDevice(&h->device);

    if (o.cuda_stream) {
        h->stream = (cudaStream_t)o.cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(nullptr, e, "cudaStreamCreate");
        }
        h->own_stream = true;
    }

    const long long maxcells = N + 1;
    h->pitch = (maxcells + 63) / 64 * 64;  // 512-byte aligned planes
    const long long planes = (long long)h->nv * h->K;
    const bool mixed = o.precision != WCC_FP64;  // FP32 planes (FP32-mixed and FP32)
    const size_t state_bytes = mixed ? (size_t)((long long)h->nv * (h->K + 1) * h->pitch) * sizeof(float)
                                     : (size_t)(planes * h->pitch) * sizeof(double);
    const size_t staging_bytes = (size_t)(maxcells * planes) * sizeof(double);
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i)
        ok = mixed ? cudaMalloc(&h->s32[i], state_bytes) == cudaSuccess
                   : cudaMalloc(&h->s64[i], state_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&h->staging, staging_bytes) == cudaSuccess &&
         cudaMalloc(&h->st, sizeof(DevState)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(h);
        delete h;
        return fail(nullptr, WCC_E_NOMEM, "cudaMalloc of the solver state failed");
    }
    h->bytes = 2 * (long long)state_bytes + (long long)staging_bytes + (long long)sizeof(DevState);
    // zero the padding once so that no plane ever holds uninitialised data
    for (int i = 0; i < 2; ++i)
        cudaMemsetAsync(mixed ? (void*)h->s32[i] : (void*)h->s64[i], 0, state_bytes, h->stream);
    cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream);
    if (ensure_history(h, 4096) != WCC_OK) {
        std::string m = h->err;
        release(h);
        delete h;
        return fail(nullptr, WCC_E_NOMEM, m);
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        release(h);
        delete h;
        return cuda_fail(nullptr, e, "wcc_create");
    }
    *out = h;
    return WCC_OK;
}

int wcc_num_cells(wcc_handle h, int64_t* ncells) {
    if (!h || !ncells) return fail(h, WCC_E_INVAL, "NULL argument");
    *ncells = stage_cells(h, h->parity);
    return WCC_OK;
}

int wcc_set_initial(wcc_handle h, const double* dofs, int64_t count) {
    WccTraceRange trace_("wcc_set_initial");
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!dofs) return fail(h, WCC_E_INVAL, "dofs is NULL");
    const long long n = stage_cells(h, 0);
    if (count != n * h->nv * h->K) return fail(h, WCC_E_INVAL, "count does not match cells*nv*(P+1) of an integer stage");
    // host -> device staging by a copy engine (overlaps kernels of other
    // streams), then the layout conversion on the device
    WCC_CHECK(h, cudaMemcpyAsync(h->staging, dofs, (size_t)count * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream));
    const double* src = h->staging;
    h->cur = 0;
    h->parity = 0;
    h->steps = 0;
    h->tb_pairs = h->tb_fallbacks = 0;
    const bool mixed = h->opt.precision != WCC_FP64;
    WCC_CHECK(h, cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
    StepArgs a = make_args(h, 0, 0, 0.0, 0.0);
    cudaError_t e;
    if (mixed) {
        // conversion and the stage's CFL bound in one kernel
        const int keep_lo = h->opt.precision == WCC_FP32_MIXED;
        switch (h->system) {
            case WCC_ADVECTION: e = launch_load_stage_mixed<ADVECTION>(h->P, src, n, h->pitch, h->s32[0], keep_lo, a, 0, h->stream); break;
            case WCC_BURGERS: e = launch_load_stage_mixed<BURGERS>(h->P, src, n, h->pitch, h->s32[0], keep_lo, a, 0, h->stream); break;
            default: e = launch_load_stage_mixed<EULER>(h->P, src, n, h->pitch, h->s32[0], keep_lo, a, 0, h->stream); break;
        }
        h->launches += 1;
    } else {
        aos_to_planes_fp64<<<conv_grid(n), kConvThreads, 0, h->stream>>>(src, n, h->nv, h->K, h->pitch,
                                                                              h->s64[0]);
        WCC_CHECK(h, cudaGetLastError());
        const long long var_stride = (long long)h->K * h->pitch;
        switch (h->system) {
            case WCC_ADVECTION: e = launch_stage_speed<ADVECTION>(h->s64[0], var_stride, n, a, 0, h->stream); break;
            case WCC_BURGERS: e = launch_stage_speed<BURGERS>(h->s64[0], var_stride, n, a, 0, h->stream); break;
            default: e = launch_stage_speed<EULER>(h->s64[0], var_stride, n, a, 0, h->stream); break;
        }
        h->launches += 2;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "stage set-up launch");
    h->initialised = true;
    DevState s;
    int rc = read_state(h, &s);
    if (rc != WCC_OK) {
        h->initialised = false;
        return rc;
    }
    return WCC_OK;
}

}  // extern "C"

namespace {
// A CFL number must be positive and at most the degree's linear stability
// limit (Sec. 2.3, Table 1; wcc_stability_limit).
int check_cfl(wcc_ctx* h, double cfl) {
    if (!(cfl > 0.0) || !(cfl < 1e6)) return fail(h, WCC_E_INVAL, "cfl must be a positive number");
    double lim = 0.0;
    if (wcc_stability_limit(h->P, &lim) == WCC_OK && cfl > lim)
        return fail(h, WCC_E_CFL, "cfl above the linear stability limit of the degree (wcc_stability_limit)");
    return WCC_OK;
}
}  // namespace

extern "C" {

int wcc_step(wcc_handle h, int64_t nsteps, double cfl) {
    WccTraceRange trace_("wcc_step");
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!h->initialised) return fail(h, WCC_E_STATE, "wcc_set_initial has not been called");
    if (nsteps < 0) return fail(h, WCC_E_INVAL, "nsteps < 0");
    int rc = check_cfl(h, cfl);
    if (rc != WCC_OK) return rc;
    rc = ensure_history(h, h->steps + nsteps);
    if (rc != WCC_OK) return rc;
    if (h->opt.tb_depth == 2) return step_pairs(h, nsteps, cfl);
    return step_single(h, nsteps, cfl);
}

int wcc_tb_stats(wcc_handle h, int64_t* pairs, int64_t* fallbacks, double* nu2_max) {
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    DevState s;
    int rc = read_state(h, &s);
    if (pairs) *pairs = h->tb_pairs;
    if (fallbacks) *fallbacks = h->tb_fallbacks;
    if (nu2_max) *nu2_max = s.tb_nu2_max;
    return rc;
}

int wcc_autotune(wcc_handle h, double cfl, int* cells_per_block, int* tb_depth) {
    WccTraceRange trace_("wcc_autotune");
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!h->initialised) return fail(h, WCC_E_STATE, "wcc_set_initial has not been called");
    if (int rc = check_cfl(h, cfl)) return rc;
    struct Cand {
        int cpb, tb;
    };
    Cand cands[3];
    int nc = 0;
    if (h->opt.precision == WCC_FP32_MIXED) {
        cands[nc++] = {kTileMixed, 1};
        cands[nc++] = {2 * kTileMixed, 1};
        cands[nc++] = {0, 2};
    }
    const wcc_options saved = h->opt;
    if (nc == 0) {  // one compiled configuration
        if (cells_per_block) *cells_per_block = saved.cells_per_block;
        if (tb_depth) *tb_depth = saved.tb_depth;
        return WCC_OK;
    }
    const int chunk = h->opt.graph_chunk >= 2 ? h->opt.graph_chunk : 32;
    int rc = ensure_history(h, h->steps + 4 * chunk + 2);
    if (rc != WCC_OK) return rc;
    // the state to return to: the current stage, the device state, the
    // host-side position and the pair counters
    DevState st0;
    if ((rc = read_state(h, &st0)) != WCC_OK) return rc;
    if (h->tb_limit == 0.0 && wcc_stability_limit(h->P, &h->tb_limit) != WCC_OK)
        return fail(h, WCC_E_INVAL, "no stability limit for this P");
    const int cur0 = h->cur, parity0 = h->parity;
    const long long steps0 = h->steps, pairs0 = h->tb_pairs, fb0 = h->tb_fallbacks;
    const size_t bytes = (size_t)((long long)h->nv * (h->K + 1) * h->pitch) * sizeof(float);
    float* copy = nullptr;
    if (cudaMalloc(&copy, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, WCC_E_NOMEM, "cudaMalloc of the autotuner's stage copy failed");
    }
    auto restore = [&]() -> int {
        WCC_CHECK(h, cudaMemcpyAsync(h->s32[cur0], copy, bytes, cudaMemcpyDeviceToDevice, h->stream));
        WCC_CHECK(h, cudaMemcpyAsync(h->st, &st0, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
        WCC_CHECK(h, cudaStreamSynchronize(h->stream));
        h->cur = cur0;
        h->parity = parity0;
        h->steps = steps0;
        h->tb_pairs = pairs0;
        h->tb_fallbacks = fb0;
        return WCC_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best_ms = 0.f;
    int best = -1;
    rc = cudaMemcpyAsync(copy, h->s32[cur0], bytes, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess &&
                 cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess
             ? WCC_OK
             : cuda_fail(h, cudaGetLastError(), "autotuner set-up");
    for (int i = 0; i < nc && rc == WCC_OK; ++i) {
        h->opt.cells_per_block = cands[i].cpb;
        h->opt.tb_depth = cands[i].tb;
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        if ((rc = restore()) != WCC_OK) break;
        if ((rc = wcc_step(h, chunk, cfl)) != WCC_OK) break;  // warm-up (and graph capture)
        DevState warm;
        if ((rc = read_state(h, &warm)) != WCC_OK) break;
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < 3 && rc == WCC_OK; ++r) rc = wcc_step(h, chunk, cfl);
        cudaEventRecord(e1, h->stream);
        if (rc != WCC_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = cuda_fail(h, cudaGetLastError(), "autotuner timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0 || ms < best_ms) {
            best_ms = ms;
            best = i;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->opt = saved;
    if (best >= 0 && rc == WCC_OK) {
        h->opt.cells_per_block = cands[best].cpb;
        h->opt.tb_depth = cands[best].tb;
    }
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    const int rrc = restore();
    cudaFree(copy);
    if (rc != WCC_OK) return rc;
    if (rrc != WCC_OK) return rrc;
    if (cells_per_block) *cells_per_block = h->opt.cells_per_block;
    if (tb_depth) *tb_depth = h->opt.tb_depth;
    return WCC_OK;
}

int wcc_step_dt(wcc_handle h, int64_t nsteps, const double* dts) {
    WccTraceRange trace_("wcc_step_dt");
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!h->initialised) return fail(h, WCC_E_STATE, "wcc_set_initial has not been called");
    if (nsteps < 0 || (nsteps > 0 && !dts)) return fail(h, WCC_E_INVAL, "bad nsteps / dts");
    for (int64_t s = 0; s < nsteps; ++s)
        if (!(dts[s] > 0.0) || !(dts[s] < 1e300)) return fail(h, WCC_E_INVAL, "every dt must be positive and finite");
    int rc = ensure_history(h, h->steps + nsteps);
    if (rc != WCC_OK) return rc;
    for (int64_t s = 0; s < nsteps; ++s) {
        rc = enqueue_one(h, 0.0, dts[s]);
        if (rc != WCC_OK) return rc;
    }
    return WCC_OK;
}

int wcc_get_dofs(wcc_handle h, double* dofs, int64_t count) {
    WccTraceRange trace_("wcc_get_dofs");
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!dofs) return fail(h, WCC_E_INVAL, "dofs is NULL");
    if (!h->initialised) return fail(h, WCC_E_STATE, "wcc_set_initial has not been called");
    const long long n = stage_cells(h, h->parity);
    if (count != n * h->nv * h->K) return fail(h, WCC_E_INVAL, "count does not match the current stage");
    if (h->opt.precision != WCC_FP64) {
        WCC_CHECK(h, launch_planes_to_aos_mixed(h->K, conv_grid(n), h->stream, h->s32[h->cur], n, h->nv, h->pitch,
                                                h->staging));
    } else {
        planes_to_aos_fp64<<<conv_grid(n), kConvThreads, 0, h->stream>>>(h->s64[h->cur], n, h->nv, h->K, h->pitch,
                                                                        h->staging);
        WCC_CHECK(h, cudaGetLastError());
    }
    h->launches += 1;
    WCC_CHECK(h, cudaMemcpyAsync(dofs, h->staging, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    DevState s;
    return read_state(h, &s);
}

int wcc_step_until(wcc_handle h, double t_end, double cfl, int64_t* nsteps_taken) {
    WccTraceRange trace_("wcc_step_until");
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (nsteps_taken) *nsteps_taken = 0;
    if (!h->initialised) return fail(h, WCC_E_STATE, "wcc_set_initial has not been called");
    if (int rc = check_cfl(h, cfl)) return rc;
    if (!(std::fabs(t_end) < 1e300)) return fail(h, WCC_E_INVAL, "t_end must be finite");
    if (h->parity != 0) return fail(h, WCC_E_STATE, "wcc_step_until starts on an integer stage");
    DevState s;
    int rc = read_state(h, &s);
    if (rc != WCC_OK) return rc;
    if (t_end < s.t) return fail(h, WCC_E_INVAL, "t_end is before the current time");
    const unsigned long long cfl_bits = (unsigned long long)__double_as_longlong_host(cfl);
    // the size the next CFL half-step will take: the kernels' own rule
    auto next_dt = [&](const DevState& st) {
        if ((unsigned long long)__double_as_longlong_host(st.next_cfl) == cfl_bits) return st.next_dt;
        double amax;
        std::memcpy(&amax, &st.amax_bits[h->parity], sizeof amax);
        return cfl * h->dx / amax;
    };
    int64_t taken = 0;
    auto finish = [&](int code) {
        if (nsteps_taken) *nsteps_taken = taken;
        return code;
    };
    const int chunk = h->opt.graph_chunk >= 2 ? h->opt.graph_chunk : 2;
    for (;;) {
        const double dt = next_dt(s);
        if (!(dt > 0.0) || !(dt < 1e300)) return finish(fail(h, WCC_E_NONFINITE, "the CFL half-step size is not positive"));
        const double left = t_end - s.t;
        // a rest below 1e-9 of a half-step is the rounding of the summed time
        const double tiny = std::max(1e-14 * std::max(1.0, std::fabs(t_end)), 1e-9 * dt);
        if (left >= 4.0 * chunk * dt) {  // far from t_end: a whole graph (dt may grow a little)
            if ((rc = wcc_step(h, chunk, cfl)) != WCC_OK) return finish(rc);
            taken += chunk;
        } else if (left >= 2.0 * dt * (1.0 - 1e-12)) {  // a pair of CFL half-steps fits
            if ((rc = wcc_step(h, 1, cfl)) != WCC_OK) return finish(rc);
            ++taken;
            if ((rc = read_state(h, &s)) != WCC_OK) return finish(rc);
            const double left2 = t_end - s.t;
            if (left2 >= next_dt(s) * (1.0 - 1e-12)) {
                if ((rc = wcc_step(h, 1, cfl)) != WCC_OK) return finish(rc);
            } else {  // the second CFL step would pass t_end
                if ((rc = wcc_step_dt(h, 1, &left2)) != WCC_OK) return finish(rc);
            }
            ++taken;
        } else {  // the rest, in two equal half-steps
            if (left > tiny) {
                const double dts[2] = {0.5 * left, 0.5 * left};
                if ((rc = wcc_step_dt(h, 2, dts)) != WCC_OK) return finish(rc);
                taken += 2;
            }
            break;
        }
        if ((rc = read_state(h, &s)) != WCC_OK) return finish(rc);
        if (s.t >= t_end - 1e-14 * std::max(1.0, std::fabs(t_end))) break;
    }
    return finish(read_state(h, &s));
}

int wcc_get_state(wcc_handle h, double* t, int64_t* half_steps, int* parity) {
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    DevState s;
    int rc = read_state(h, &s);
    if (t) *t = s.t;
    if (half_steps) *half_steps = s.step;
    if (parity) *parity = h->parity;
    return rc;
}

int wcc_get_dt_history(wcc_handle h, double* dts, int64_t cap, int64_t* n) {
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (cap < 0 || (cap > 0 && !dts)) return fail(h, WCC_E_INVAL, "bad dts / cap");
    DevState s;
    int rc = read_state(h, &s);
    long long taken = s.step;
    if (n) *n = taken;
    long long m = taken < cap ? taken : cap;
    if (m > h->hist_cap) m = h->hist_cap;
    if (m > 0) WCC_CHECK(h, cudaMemcpy(dts, h->hist, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost));
    return rc;
}

int wcc_synchronize(wcc_handle h) {
    if (!h) return fail(nullptr, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    DevState s;
    return read_state(h, &s);
}

int wcc_device_bytes(wcc_handle h, int64_t* bytes) {
    if (!h || !bytes) return fail(h, WCC_E_INVAL, "NULL argument");
    *bytes = h->bytes;
    return WCC_OK;
}

int wcc_launch_count(wcc_handle h, int64_t* launches) {
    if (!h || !launches) return fail(h, WCC_E_INVAL, "NULL argument");
    *launches = h->launches;
    return WCC_OK;
}

const char* wcc_last_error(wcc_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void wcc_destroy(wcc_handle h) {
    if (!h) return;
    DeviceScope ds_(h->device);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

}  // extern "C"
