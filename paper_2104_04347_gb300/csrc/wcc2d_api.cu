// wcc2d_api.cu -- the C ABI of include/wcc2d.h: handle, device memory,
// host <-> device layout conversion, the half-step loop and the CFL time
// stepping of the 2D path (Sec. 3.1: alternating integer and half stages).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "wcc.h"
#include "wcc2d.h"
#include "wcc2d_kernels.cuh"
#include "wcc_launch.h"
#include "wcc_trace.h"

using wcc::DeviceScope;
using namespace wcc2d;

namespace {
thread_local std::string g_create_error2d;
}

struct wcc2d_ctx {
    int system = 0, P = 1, bc = 0, nv = 1, nq = 3;
    int fp32 = 0;   // float storage (WCC_FP32 or WCC_FP32_MIXED)
    int mixed = 0;  // WCC_FP32_MIXED: float-float cell averages
    int device = 0;
    int64_t nx = 0, ny = 0;
    double x0 = 0, x1 = 1, y0 = 0, y1 = 1, dx = 1, dy = 1;
    wcc2d_options opt{};
    Law2D law{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* planes[2] = {nullptr, nullptr};  // stage buffers of T
    double* staging = nullptr;             // host-layout FP64 copy of a stage
    DevState2D* st = nullptr;
    double* hist = nullptr;
    long long hist_cap = 0;
    long long pitch = 0, rows_alloc = 0, plane = 0;
    int cur = 0;         // buffer holding the current stage
    int parity = 0;      // parity of the current stage
    long long steps = 0; // half-steps taken since set_initial
    bool loaded = false;
    long long launches = 0;
    long long bytes = 0;
    std::string err;
};

namespace {

int fail2(wcc2d_ctx* h, int code, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_create_error2d = msg;
    return code;
}

int cuda_fail2(wcc2d_ctx* h, cudaError_t e, const char* what) {
    return fail2(h, WCC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define WCC2D_CHECK(h, call)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail2(h, e_, #call); \
    } while (0)

int64_t stage_cells_x(const wcc2d_ctx* h, int parity) { return h->bc == WCC_BC_PERIODIC ? h->nx : h->nx + 1 - parity; }
int64_t stage_cells_y(const wcc2d_ctx* h, int parity) { return h->bc == WCC_BC_PERIODIC ? h->ny : h->ny + 1 - parity; }

size_t elem_size(const wcc2d_ctx* h) { return h->fp32 ? sizeof(float) : sizeof(double); }

void release(wcc2d_ctx* h) {
    for (int i = 0; i < 2; ++i)
        if (h->planes[i]) cudaFree(h->planes[i]);
    if (h->staging) cudaFree(h->staging);
    if (h->st) cudaFree(h->st);
    if (h->hist) cudaFree(h->hist);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int ensure_history(wcc2d_ctx* h, long long need) {
    if (need <= h->hist_cap) return WCC_OK;
    long long cap = h->hist_cap > 0 ? h->hist_cap : 4096;
    while (cap < need) cap *= 2;
    double* nh = nullptr;
    if (cudaMalloc(&nh, (size_t)cap * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail2(h, WCC_E_NOMEM, "cudaMalloc of the dt history failed");
    }
    if (h->hist) {
        WCC2D_CHECK(h, cudaMemcpyAsync(nh, h->hist, (size_t)h->hist_cap * sizeof(double), cudaMemcpyDeviceToDevice,
                                       h->stream));
        WCC2D_CHECK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->hist);
    }
    h->bytes += (cap - h->hist_cap) * (long long)sizeof(double);
    h->hist = nh;
    h->hist_cap = cap;
    return WCC_OK;
}

// Reads the device state and turns its error bits into a return code.
int read_state(wcc2d_ctx* h, DevState2D* out) {
    WCC2D_CHECK(h, cudaMemcpyAsync(out, h->st, sizeof(DevState2D), cudaMemcpyDeviceToHost, h->stream));
    WCC2D_CHECK(h, cudaStreamSynchronize(h->stream));
    if (out->err & ERR_BOUNDS) return fail2(h, WCC_E_CUDA, "bounds check failed in the half-step kernel");
    if (out->err & ERR_POSITIVITY) return fail2(h, WCC_E_POSITIVITY, "non-positive density or pressure");
    if (out->err & ERR_NONFINITE) return fail2(h, WCC_E_NONFINITE, "non-finite DOF or CFL bound");
    return WCC_OK;
}

int conv_grid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

extern "C" {

void wcc2d_default_options(wcc2d_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = WCC_FP64;
    o->limiter = 1;
    o->alpha = 2.0;
    o->eps = 1e-40;
    o->gamma = 1.4;
    o->ax = 1.0;
    o->ay = 1.0;
    o->rows_per_cta = 16;
    o->cuda_stream = nullptr;
}

int wcc2d_create(wcc2d_handle* out, int system, int64_t nx, int64_t ny, int P, const double domain[4], int bc,
                 const wcc2d_options* opt) {
    if (!out || !domain) return fail2(nullptr, WCC_E_INVAL, "NULL argument");
    *out = nullptr;
    if (system != WCC_ADVECTION && system != WCC_BURGERS && system != WCC_EULER)
        return fail2(nullptr, WCC_E_INVAL, "unknown system");
    if (P < 1 || P > 3) return fail2(nullptr, WCC_E_INVAL, "P must be 1..3");
    if (nx < 4 || ny < 4) return fail2(nullptr, WCC_E_INVAL, "nx and ny must be >= 4");
    if (nx > (1 << 15) || ny > (1 << 15)) return fail2(nullptr, WCC_E_CAPACITY, "nx and ny must be <= 2^15");
    if (bc != WCC_BC_PERIODIC && bc != WCC_BC_TRANSMISSIVE) return fail2(nullptr, WCC_E_INVAL, "unknown bc");
    if (!(domain[1] > domain[0]) || !(domain[3] > domain[2]) || !std::isfinite(domain[0]) ||
        !std::isfinite(domain[1]) || !std::isfinite(domain[2]) || !std::isfinite(domain[3]))
        return fail2(nullptr, WCC_E_INVAL, "bad domain");
    wcc2d_options o;
    if (opt)
        o = *opt;
    else
        wcc2d_default_options(&o);
    if (o.precision != WCC_FP64 && o.precision != WCC_FP32 && o.precision != WCC_FP32_MIXED)
        return fail2(nullptr, WCC_E_INVAL, "precision must be WCC_FP64, WCC_FP32_MIXED or WCC_FP32");
    if (!(o.alpha > 0) || !(o.eps >= 0) || !(o.gamma > 1) || o.rows_per_cta < 1 || o.rows_per_cta > 4096 ||
        !std::isfinite(o.ax) || !std::isfinite(o.ay))
        return fail2(nullptr, WCC_E_INVAL, "bad options");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail2(nullptr, WCC_E_CUDA, "no usable CUDA device");
    }
    wcc2d_ctx* h = new wcc2d_ctx();
    cudaGetDevice(&h->device);
    h->system = system;
    h->P = P;
    h->bc = bc;
    h->nv = system == WCC_EULER ? 4 : 1;
    h->nq = (P + 1) * (P + 2) / 2;
    h->fp32 = o.precision != WCC_FP64;
    h->mixed = o.precision == WCC_FP32_MIXED;
    h->nx = nx;
    h->ny = ny;
    h->x0 = domain[0];
    h->x1 = domain[1];
    h->y0 = domain[2];
    h->y1 = domain[3];
    h->dx = (domain[1] - domain[0]) / (double)nx;
    h->dy = (domain[3] - domain[2]) / (double)ny;
    h->opt = o;
    h->law = Law2D{o.ax, o.ay, o.gamma, o.alpha, o.eps, o.limiter ? 1 : 0};
    if (o.cuda_stream) {
        h->stream = static_cast<cudaStream_t>(o.cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail2(nullptr, WCC_E_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    const long long maxx = nx + 1, maxy = ny + 1;
    const long long align = h->fp32 ? 32 : 16;  // 128-byte aligned rows
    h->pitch = (maxx + align - 1) / align * align;
    h->rows_alloc = maxy;
    h->plane = h->pitch * h->rows_alloc;
    // FP32-mixed: one more plane per variable for the low part of the average
    const size_t stage_bytes = (size_t)(h->nv * (h->nq + (h->mixed ? 1 : 0))) * (size_t)h->plane * elem_size(h);
    const size_t staging_bytes = (size_t)(maxx * maxy) * (size_t)(h->nv * h->nq) * sizeof(double);
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) ok = cudaMalloc(&h->planes[i], stage_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&h->staging, staging_bytes) == cudaSuccess &&
         cudaMalloc(&h->st, sizeof(DevState2D)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(h);
        delete h;
        return fail2(nullptr, WCC_E_NOMEM, "cudaMalloc of the 2D solver state failed");
    }
    h->bytes = 2 * (long long)stage_bytes + (long long)staging_bytes + (long long)sizeof(DevState2D);
    for (int i = 0; i < 2; ++i) cudaMemsetAsync(h->planes[i], 0, stage_bytes, h->stream);
    cudaMemsetAsync(h->st, 0, sizeof(DevState2D), h->stream);
    if (ensure_history(h, 4096) != WCC_OK) {
        std::string m = h->err;
        release(h);
        delete h;
        return fail2(nullptr, WCC_E_NOMEM, m);
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        release(h);
        delete h;
        return cuda_fail2(nullptr, e, "wcc2d_create");
    }
    *out = h;
    return WCC_OK;
}

int wcc2d_destroy(wcc2d_handle h) {
    if (!h) return WCC_OK;
    {
        DeviceScope ds_(h->device);
        if (h->stream) cudaStreamSynchronize(h->stream);
        release(h);
    }
    delete h;
    return WCC_OK;
}

const char* wcc2d_last_error(wcc2d_handle h) { return h ? h->err.c_str() : g_create_error2d.c_str(); }

int wcc2d_stage_dims(wcc2d_handle h, int64_t* nx, int64_t* ny) {
    if (!h || !nx || !ny) return fail2(h, WCC_E_INVAL, "NULL argument");
    *nx = stage_cells_x(h, h->parity);
    *ny = stage_cells_y(h, h->parity);
    return WCC_OK;
}

int wcc2d_set_initial(wcc2d_handle h, const double* dofs, int64_t count) {
    WccTraceRange trace_("wcc2d_set_initial");
    if (!h || !dofs) return fail2(h, WCC_E_INVAL, "NULL argument");
    DeviceScope ds_(h->device);
    const int64_t cx = stage_cells_x(h, 0), cy = stage_cells_y(h, 0);
    const int nd = h->nv * h->nq;
    if (count != cx * cy * nd) return fail2(h, WCC_E_INVAL, "count does not match an integer stage");
    WCC2D_CHECK(h, cudaMemcpyAsync(h->staging, dofs, (size_t)count * sizeof(double), cudaMemcpyHostToDevice,
                                   h->stream));
    const int g = conv_grid(cx * cy * nd);
    if (h->mixed)
        WCC2D_CHECK(h, launch_convert2d_mx(h->P, true, h->staging, static_cast<float*>(h->planes[0]), (int)cx, (int)cy,
                                           h->nv, h->pitch, h->plane, h->stream));
    else if (h->fp32)
        aos_to_planes2d<float><<<g, 256, 0, h->stream>>>(h->staging, static_cast<float*>(h->planes[0]), (int)cx,
                                                         (int)cy, nd, h->pitch, h->plane);
    else
        aos_to_planes2d<double><<<g, 256, 0, h->stream>>>(h->staging, static_cast<double*>(h->planes[0]), (int)cx,
                                                          (int)cy, nd, h->pitch, h->plane);
    WCC2D_CHECK(h, cudaGetLastError());
    WCC2D_CHECK(h, cudaMemsetAsync(h->st, 0, sizeof(DevState2D), h->stream));
    if (h->mixed)
        WCC2D_CHECK(h, launch_stage_rate2d_mx(h->system, h->P, static_cast<const float*>(h->planes[0]), h->pitch,
                                              h->plane, (int)cx, (int)cy, h->law, h->dx, h->dy, h->st, h->stream));
    else
        WCC2D_CHECK(h, launch_stage_rate2d(h->system, h->fp32, h->planes[0], h->pitch, h->plane, (int)cx, (int)cy,
                                           h->nq, h->law, h->dx, h->dy, h->st, h->stream));
    h->launches += 2;
    h->cur = 0;
    h->parity = 0;
    h->steps = 0;
    h->loaded = false;
    DevState2D s;
    int rc = read_state(h, &s);
    if (rc != WCC_OK) return rc;
    h->loaded = true;
    return WCC_OK;
}

namespace {

// Enqueue one half-step: dt_given > 0 fixes its size, otherwise the kernel
// takes cfl / (CFL rate of the current stage) from the device state.
int launch_one(wcc2d_ctx* h, double dt_given, double cfl) {
    Step2D a;
    a.in = h->planes[h->cur];
    a.out = h->planes[h->cur ^ 1];
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.rows_alloc = h->rows_alloc;
    a.nx_old = (int)stage_cells_x(h, h->parity);
    a.ny_old = (int)stage_cells_y(h, h->parity);
    a.nx_new = (int)stage_cells_x(h, h->parity ^ 1);
    a.ny_new = (int)stage_cells_y(h, h->parity ^ 1);
    a.parity = h->parity;
    a.bc = h->bc;
    a.rows_per_cta = h->opt.rows_per_cta;
    a.dx = h->dx;
    a.dy = h->dy;
    a.inv_dx = 1.0 / h->dx;
    a.inv_dy = 1.0 / h->dy;
    a.dt_given = dt_given;
    a.cfl = cfl;
    a.law = h->law;
    a.st = h->st;
    a.hist = h->hist;
    a.hist_cap = h->hist_cap;
    cudaError_t e = h->mixed ? launch_halfstep2d_mx(h->system, h->P, a, h->stream)
                             : launch_halfstep2d(h->system, h->P, h->fp32 != 0, a, h->stream);
    if (e != cudaSuccess) return cuda_fail2(h, e, "2D half-step launch");
    h->cur ^= 1;
    h->parity ^= 1;
    h->steps += 1;
    h->launches += 1;
    return WCC_OK;
}

// The CFL half-step the kernels will take on the stage of this parity (the
// same double expression as in the kernel).
double cfl_dt_of(const DevState2D& s, int parity, double cfl) {
    double rate;
    std::memcpy(&rate, &s.rate_bits[parity], sizeof(rate));
    return cfl / rate;
}

}  // namespace

int wcc2d_step(wcc2d_handle h, int64_t nsteps, double cfl) {
    WccTraceRange trace_("wcc2d_step");
    if (!h) return fail2(h, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!h->loaded) return fail2(h, WCC_E_STATE, "wcc2d_set_initial has not succeeded");
    if (nsteps < 0 || !(cfl > 0) || !std::isfinite(cfl)) return fail2(h, WCC_E_INVAL, "bad nsteps or cfl");
    int rc = ensure_history(h, h->steps + nsteps);
    if (rc != WCC_OK) return rc;
    for (int64_t i = 0; i < nsteps; ++i)
        if ((rc = launch_one(h, 0.0, cfl)) != WCC_OK) return rc;
    return WCC_OK;
}

int wcc2d_step_dt(wcc2d_handle h, int64_t nsteps, const double* dts) {
    WccTraceRange trace_("wcc2d_step_dt");
    if (!h) return fail2(h, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!h->loaded) return fail2(h, WCC_E_STATE, "wcc2d_set_initial has not succeeded");
    if (nsteps < 0 || (nsteps > 0 && !dts)) return fail2(h, WCC_E_INVAL, "bad nsteps or dts");
    for (int64_t i = 0; i < nsteps; ++i)
        if (!(dts[i] > 0) || !std::isfinite(dts[i])) return fail2(h, WCC_E_INVAL, "dt must be finite and > 0");
    int rc = ensure_history(h, h->steps + nsteps);
    if (rc != WCC_OK) return rc;
    for (int64_t i = 0; i < nsteps; ++i)
        if ((rc = launch_one(h, dts[i], 0.0)) != WCC_OK) return rc;
    return WCC_OK;
}

int wcc2d_step_until(wcc2d_handle h, double t_end, double cfl, int64_t* nsteps_taken) {
    WccTraceRange trace_("wcc2d_step_until");
    if (!h) return fail2(h, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (nsteps_taken) *nsteps_taken = 0;
    if (!h->loaded) return fail2(h, WCC_E_STATE, "wcc2d_set_initial has not succeeded");
    if (h->parity != 0) return fail2(h, WCC_E_STATE, "wcc2d_step_until starts on an integer stage");
    if (!std::isfinite(t_end) || !(cfl > 0) || !std::isfinite(cfl)) return fail2(h, WCC_E_INVAL, "bad t_end or cfl");
    DevState2D s;
    int rc = read_state(h, &s);
    if (rc != WCC_OK) return rc;
    const double scale = std::max(1.0, std::fabs(t_end));
    if (t_end < s.t - 1e-14 * scale) return fail2(h, WCC_E_INVAL, "t_end is before the current time");
    const int chunk = 32;
    int64_t taken = 0;
    for (;;) {
        const double left = t_end - s.t;
        if (left <= 1e-14 * scale) break;
        const double dt = cfl_dt_of(s, h->parity, cfl);
        if (!(dt > 0) || !std::isfinite(dt)) return fail2(h, WCC_E_NONFINITE, "non-finite CFL step");
        const double tiny = std::max(1e-14 * scale, 1e-9 * dt);
        if (left >= 4.0 * chunk * dt) {
            // far from t_end the CFL bound cannot change enough to matter
            if ((rc = wcc2d_step(h, chunk, cfl)) != WCC_OK) return rc;
            taken += chunk;
        } else if (left >= 2.0 * dt * (1.0 - 1e-12)) {
            if ((rc = ensure_history(h, h->steps + 2)) != WCC_OK) return rc;
            if ((rc = launch_one(h, 0.0, cfl)) != WCC_OK) return rc;
            if ((rc = read_state(h, &s)) != WCC_OK) return rc;
            const double left2 = t_end - s.t;
            const double dt2 = cfl_dt_of(s, h->parity, cfl);
            if (!(dt2 > 0) || !std::isfinite(dt2)) return fail2(h, WCC_E_NONFINITE, "non-finite CFL step");
            if (left2 >= dt2 * (1.0 - 1e-12)) {
                if ((rc = launch_one(h, 0.0, cfl)) != WCC_OK) return rc;
            } else {
                if ((rc = launch_one(h, left2, 0.0)) != WCC_OK) return rc;
                taken += 2;
                if ((rc = read_state(h, &s)) != WCC_OK) return rc;
                break;
            }
            taken += 2;
        } else {
            if (left > tiny) {
                if ((rc = ensure_history(h, h->steps + 2)) != WCC_OK) return rc;
                if ((rc = launch_one(h, 0.5 * left, 0.0)) != WCC_OK) return rc;
                if ((rc = launch_one(h, 0.5 * left, 0.0)) != WCC_OK) return rc;
                taken += 2;
            }
            if ((rc = read_state(h, &s)) != WCC_OK) return rc;
            break;
        }
        if ((rc = read_state(h, &s)) != WCC_OK) return rc;
    }
    if (nsteps_taken) *nsteps_taken = taken;
    return WCC_OK;
}

int wcc2d_get_dofs(wcc2d_handle h, double* dofs, int64_t count) {
    WccTraceRange trace_("wcc2d_get_dofs");
    if (!h || !dofs) return fail2(h, WCC_E_INVAL, "NULL argument");
    DeviceScope ds_(h->device);
    if (!h->loaded) return fail2(h, WCC_E_STATE, "wcc2d_set_initial has not succeeded");
    const int64_t cx = stage_cells_x(h, h->parity), cy = stage_cells_y(h, h->parity);
    const int nd = h->nv * h->nq;
    if (count != cx * cy * nd) return fail2(h, WCC_E_INVAL, "count does not match the current stage");
    DevState2D s;
    int rc = read_state(h, &s);
    if (rc != WCC_OK) return rc;
    const int g = conv_grid(cx * cy * nd);
    if (h->mixed)
        WCC2D_CHECK(h, launch_convert2d_mx(h->P, false, h->staging, static_cast<float*>(h->planes[h->cur]), (int)cx,
                                           (int)cy, h->nv, h->pitch, h->plane, h->stream));
    else if (h->fp32)
        planes_to_aos2d<float><<<g, 256, 0, h->stream>>>(static_cast<const float*>(h->planes[h->cur]), h->staging,
                                                         (int)cx, (int)cy, nd, h->pitch, h->plane);
    else
        planes_to_aos2d<double><<<g, 256, 0, h->stream>>>(static_cast<const double*>(h->planes[h->cur]), h->staging,
                                                          (int)cx, (int)cy, nd, h->pitch, h->plane);
    WCC2D_CHECK(h, cudaGetLastError());
    h->launches += 1;
    WCC2D_CHECK(h, cudaMemcpyAsync(dofs, h->staging, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost,
                                   h->stream));
    WCC2D_CHECK(h, cudaStreamSynchronize(h->stream));
    return WCC_OK;
}

int wcc2d_get_state(wcc2d_handle h, double* t, int64_t* steps, int* parity) {
    if (!h) return fail2(h, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    DevState2D s;
    int rc = read_state(h, &s);
    if (rc != WCC_OK) return rc;
    if (t) *t = s.t;
    if (steps) *steps = s.step;
    if (parity) *parity = h->parity;
    return WCC_OK;
}

int wcc2d_get_dt_history(wcc2d_handle h, double* dts, int64_t cap, int64_t* n) {
    if (!h) return fail2(nullptr, WCC_E_INVAL, "NULL handle");
    if (cap < 0 || (cap > 0 && !dts)) return fail2(h, WCC_E_INVAL, "bad dts / cap");
    DeviceScope ds_(h->device);
    DevState2D s;
    int rc = read_state(h, &s);
    if (n) *n = s.step;
    long long m = std::min<long long>(std::min<long long>(s.step, cap), h->hist_cap);
    if (m > 0)
        WCC2D_CHECK(h, cudaMemcpy(dts, h->hist, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost));
    return rc;
}

int wcc2d_autotune(wcc2d_handle h, double cfl, int* rows_per_cta) {
    WccTraceRange trace_("wcc2d_autotune");
    if (!h) return fail2(h, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    if (!h->loaded) return fail2(h, WCC_E_STATE, "wcc2d_set_initial has not succeeded");
    if (!(cfl > 0) || !std::isfinite(cfl)) return fail2(h, WCC_E_INVAL, "bad cfl");
    // Strip heights around the measured optimum: the number of CTAs, and so
    // how full the last wave of resident CTAs is, changes with the height.
    static const int kRows[] = {8, 10, 12, 13, 14, 15, 16, 17, 18, 19, 20, 22, 24};
    constexpr int kWarm = 1, kTimed = 4;
    const size_t stage_bytes = (size_t)(h->nv * (h->nq + (h->mixed ? 1 : 0))) * (size_t)h->plane * elem_size(h);
    int rc = ensure_history(h, h->steps + kWarm + kTimed);
    if (rc != WCC_OK) return rc;
    void* save = nullptr;
    if (cudaMalloc(&save, stage_bytes + sizeof(DevState2D)) != cudaSuccess) {
        cudaGetLastError();
        return fail2(h, WCC_E_NOMEM, "cudaMalloc of the stage copy failed");
    }
    char* sv = static_cast<char*>(save);
    const int cur0 = h->cur, parity0 = h->parity, rows0 = h->opt.rows_per_cta;
    const long long steps0 = h->steps;
    cudaMemcpyAsync(sv, h->planes[cur0], stage_bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(sv + stage_bytes, h->st, sizeof(DevState2D), cudaMemcpyDeviceToDevice, h->stream);
    auto restore = [&]() {
        cudaMemcpyAsync(h->planes[cur0], sv, stage_bytes, cudaMemcpyDeviceToDevice, h->stream);
        cudaMemcpyAsync(h->st, sv + stage_bytes, sizeof(DevState2D), cudaMemcpyDeviceToDevice, h->stream);
        h->cur = cur0;
        h->parity = parity0;
        h->steps = steps0;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_rows = rows0;
    for (int rows : kRows) {
        h->opt.rows_per_cta = rows;
        for (int k = 0; k < kWarm + kTimed && rc == WCC_OK; ++k) {
            if (k == kWarm) cudaEventRecord(e0, h->stream);
            rc = launch_one(h, 0.0, cfl);
        }
        cudaEventRecord(e1, h->stream);
        if (rc != WCC_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail2(h, WCC_E_CUDA, "autotune: a timed half-step failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_rows = rows;
        }
        restore();
    }
    if (rc != WCC_OK) restore();
    h->opt.rows_per_cta = rc == WCC_OK ? best_rows : rows0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t se = cudaStreamSynchronize(h->stream);
    cudaFree(save);
    if (rc != WCC_OK) return rc;
    if (se != cudaSuccess) return cuda_fail2(h, se, "autotune");
    if (rows_per_cta) *rows_per_cta = best_rows;
    DevState2D s;
    return read_state(h, &s);
}

int wcc2d_synchronize(wcc2d_handle h) {
    if (!h) return fail2(h, WCC_E_INVAL, "NULL handle");
    DeviceScope ds_(h->device);
    DevState2D s;
    return read_state(h, &s);
}

int wcc2d_launch_count(wcc2d_handle h, int64_t* n) {
    if (!h || !n) return fail2(h, WCC_E_INVAL, "NULL argument");
    *n = h->launches;
    return WCC_OK;
}

int wcc2d_device_bytes(wcc2d_handle h, int64_t* bytes) {
    if (!h || !bytes) return fail2(h, WCC_E_INVAL, "NULL argument");
    *bytes = h->bytes;
    return WCC_OK;
}

}  // extern "C"
