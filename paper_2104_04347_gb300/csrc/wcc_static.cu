// wcc_static.cu -- allocation-free entry point wcc_advance_static.
//
// Some callers cannot allocate device memory at the time they want to step
// a solution: a host application whose own allocator owns the whole device
// memory pool, or a code path that must not make the implicit device-wide
// synchronisation a cudaMalloc / cudaFree can cause.  For them this entry
// point runs the same FP64 half-step kernels as wcc_step on stage buffers the
// caller already owns, and keeps the kernels' scratch -- the CFL accumulators,
// counters, error bits and the dt history -- in a fixed array in the
// library's device image instead of in cudaMalloc'd memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/wcc.h"
#include "wcc_launch.h"
#include "wcc_scheme.cuh"

using namespace wcc;

namespace {

// Scratch of the allocation-free entry point: the device state followed by
// the dt history.  Every device that loads the library holds it until the
// process exits.  All calls share it.
struct StaticScratch {
    DevState st;
    double pad[(256 - sizeof(DevState) % 256) / sizeof(double)];
    double hist[WCC_STATIC_MAX_HALFSTEPS];
};

static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (driver entry
// points cuCtxGetCurrent / cuCtxGetId, reached through the runtime without
// linking the driver library), or 0 when none is current or the driver
// lacks them.  A device reset destroys the context, and the next one gets a
// new id.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device, looked up with
// that device current at the first call on it, and again whenever the
// device's context has changed since (after a cudaDeviceReset the module is
// loaded anew and the array may move).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WCC_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WCC_E_CAPACITY;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) return WCC_E_CUDA;
        g_scratch_ptr[dev] = ptr;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_ptr[dev];
    return WCC_OK;
}

long long cells_of(int bc, long long N, int parity) {
    if (bc == WCC_BC_PERIODIC) return N;
    return parity == 0 ? N + 1 : N;
}

cudaError_t step_kernel(int system, int P, const StepArgs& a, cudaStream_t s) {
    switch (system) {
        case WCC_ADVECTION: return launch_halfstep<ADVECTION>(P, PREC_FP64, a, s);
        case WCC_BURGERS: return launch_halfstep<BURGERS>(P, PREC_FP64, a, s);
        default: return launch_halfstep<EULER>(P, PREC_FP64, a, s);
    }
}

cudaError_t speed_kernel(int system, const double* planes, long long var_stride, long long n, const StepArgs& a,
                         int slot, cudaStream_t s) {
    switch (system) {
        case WCC_ADVECTION: return launch_stage_speed<ADVECTION>(planes, var_stride, n, a, slot, s);
        case WCC_BURGERS: return launch_stage_speed<BURGERS>(planes, var_stride, n, a, slot, s);
        default: return launch_stage_speed<EULER>(planes, var_stride, n, a, slot, s);
    }
}

}  // namespace

extern "C" int wcc_advance_static(int system, int P, int bc, int64_t N, const double domain[2],
                                  const wcc_options* opt, int parity, double* stage_a, double* stage_b,
                                  int64_t pitch, int64_t nsteps, double cfl, double* dts_out) {
    if (system < WCC_ADVECTION || system > WCC_EULER || P < 1 || P > 6) return WCC_E_INVAL;
    if (bc != WCC_BC_PERIODIC && bc != WCC_BC_TRANSMISSIVE) return WCC_E_INVAL;
    if (N < 4 || N > (1ll << 31) || !domain || !(domain[1] > domain[0]) || (parity != 0 && parity != 1))
        return WCC_E_INVAL;
    if (!stage_a || !stage_b || stage_a == stage_b) return WCC_E_INVAL;
    if (nsteps < 0 || !(cfl > 0.0) || !(cfl < 1e6)) return WCC_E_INVAL;
    double nu_limit = 0.0;
    if (wcc_stability_limit(P, &nu_limit) == WCC_OK && cfl > nu_limit) return WCC_E_CFL;
    if (nsteps > WCC_STATIC_MAX_HALFSTEPS) return WCC_E_CAPACITY;
    if (pitch < N + 1 || (((uintptr_t)stage_a | (uintptr_t)stage_b) & 7u)) return WCC_E_INVAL;
    wcc_options o;
    wcc_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != WCC_FP64) return WCC_E_INVAL;
    if (!(o.eps >= 0.0) || !(o.alpha > 0.0) || !(o.gamma > 1.0)) return WCC_E_INVAL;

    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != WCC_OK) return rc;
    StaticScratch* sc = static_cast<StaticScratch*>(scratch);
    cudaStream_t stream = (cudaStream_t)o.cuda_stream;

    StepArgs a{};
    a.pitch = pitch;
    a.bc = bc;
    a.limiter = o.limiter;
    a.alpha_is_two = (o.alpha == 2.0);
    a.dx = (domain[1] - domain[0]) / (double)N;
    a.cfl = cfl;
    a.cfl_mode = 1;
    a.cfl_bits = (unsigned long long)__double_as_longlong_host(cfl);
    a.adv = o.adv_speed;
    a.gamma = o.gamma;
    a.alpha = o.alpha;
    a.eps = o.eps;
    a.st = &sc->st;
    a.hist = sc->hist;
    a.hist_cap = WCC_STATIC_MAX_HALFSTEPS;

    // The array keeps the previous call's contents: clear the device state.
    if (cudaMemsetAsync(&sc->st, 0, sizeof(DevState), stream) != cudaSuccess) return WCC_E_CUDA;
    double* bufs[2] = {stage_a, stage_b};
    const long long n0 = cells_of(bc, N, parity);
    if (speed_kernel(system, stage_a, (long long)(P + 1) * pitch, n0, a, parity, stream) != cudaSuccess)
        return WCC_E_CUDA;
    int cur = 0, par = parity;
    for (int64_t s = 0; s < nsteps; ++s) {
        a.in64 = bufs[cur];
        a.out64 = bufs[cur ^ 1];
        a.parity = par;
        a.n_old = cells_of(bc, N, par);
        a.n_new = cells_of(bc, N, par ^ 1);
        if (step_kernel(system, P, a, stream) != cudaSuccess) return WCC_E_CUDA;
        cur ^= 1;
        par ^= 1;
    }
    DevState st;
    if (cudaMemcpyAsync(&st, &sc->st, sizeof(DevState), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return WCC_E_CUDA;
    if (dts_out && nsteps > 0 &&
        cudaMemcpyAsync(dts_out, sc->hist, (size_t)nsteps * sizeof(double), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess)
        return WCC_E_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return WCC_E_CUDA;
    if (st.err & ERR_POSITIVITY) return WCC_E_POSITIVITY;
    if (st.err & ERR_NONFINITE) return WCC_E_NONFINITE;
    return WCC_OK;
}
