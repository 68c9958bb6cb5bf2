/*
 * wcc.h -- C ABI of the GB300 (sm_103a) implementation of the 1D weighted
 * compact central (WCC) scheme of Shen & Parsani, "A class of high-order
 * weighted compact central schemes for solving hyperbolic conservation laws"
 * (arXiv 2104.04347), for u_t + f(u)_x = 0 with
 *   f = a u (linear advection), f = u^2/2 (Burgers), or the 1D Euler
 *   equations U = (rho, rho u, rho e), F = (rho u, rho u^2 + p, (rho e + p) u),
 *   p = (gamma - 1)(rho e - rho u^2 / 2)            (Sec. 2.1 Eq. 1DHCL; Sec. 5.2)
 *
 * Every function returns WCC_OK (0) or a negative WCC_E_* code; the message
 * of the last failure on a handle is returned by wcc_last_error(handle)
 * (wcc_last_error(NULL) for failures of wcc_create itself).  No function
 * has a CPU fallback: without a usable CUDA device every call that needs
 * one returns WCC_E_CUDA.
 *
 * Units and layout shared by all calls:
 *   - A "stage" is the set of cells at one time level.  Integer stages
 *     (t^n) hold cells centred on x_L + i dx, half stages (t^{n+1/2}) cells
 *     centred on x_L + (i + 1/2) dx, dx = (x_R - x_L)/N (Sec. 2.1, Fig. 1).
 *     Periodic: N cells per stage.  Transmissive ("non-reflection", Sec. 5.2):
 *     N+1 cells on integer stages, N on half stages; the ghost staggered
 *     cells are copies of the adjacent cell.
 *   - DOF arrays on the host side of this ABI are FP64 [cell][var][k],
 *     k = 0..P, holding the paper's scaled derivatives u_kx = dx^k d^k u/dx^k
 *     at the cell centre (Eq. 1D_Derivative_DEF, Eq. 1DPolynomial_Space),
 *     in conserved variables.  count = cells * nv * (P+1), nv = 1 or 3.
 *   - Time steps are HALF steps: one wcc_step half-step advances a stage to
 *     the next staggered stage, dt = t^{n+1/2} - t^n (Eq. 1DFlux), and the
 *     CFL number is nu = a_max dt / dx (Table 1 caption).
 *   - The device layout is private (planes [var][k][cell] of Taylor
 *     coefficients u_kx / k!, FP64 or FP32-mixed).
 *
 * Ownership: the handle owns all device memory it allocates (cudaMalloc in
 * wcc_create); caller buffers are borrowed for the duration of a call only.
 * Calls on one handle are not thread-safe, but a handle (single-grid or
 * batch) may be used from any host thread, one at a time: each call makes
 * the device the handle was created on current for its duration and then
 * restores the calling thread's device.  wcc_step only enqueues work on
 * the handle's stream; device-side errors (non-finite values, non-positive
 * density or pressure) are reported by the next call that synchronises
 * (wcc_synchronize, wcc_get_*).
 */
#ifndef WCC_H
#define WCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { WCC_ADVECTION = 0, WCC_BURGERS = 1, WCC_EULER = 2 };
enum { WCC_BC_PERIODIC = 0, WCC_BC_TRANSMISSIVE = 1 };
/* WCC_FP64: everything in double.  WCC_FP32_MIXED: FP32 Taylor coefficients
 * and FP32 arithmetic, with the cell averages, the leading flux term and the
 * vertex values in compensated FP32 (float-float).  WCC_FP32: the same
 * kernel without the compensation (the cell average rounded to one float),
 * kept to measure what the compensation buys. */
enum { WCC_FP64 = 0, WCC_FP32_MIXED = 1, WCC_FP32 = 2 };

enum {
    WCC_OK = 0,
    WCC_E_INVAL = -1,      /* bad argument (system, N, P, domain, bc, count, pointer) */
    WCC_E_STATE = -2,      /* call out of order (e.g. wcc_step before wcc_set_initial) */
    WCC_E_NOMEM = -3,      /* device or host allocation failed */
    WCC_E_CUDA = -4,       /* CUDA runtime error (no device, launch failure, ...) */
    WCC_E_NONFINITE = -5,  /* a new DOF or the CFL bound became NaN / Inf */
    WCC_E_POSITIVITY = -6, /* Euler: non-positive density or pressure at a cell centre */
    WCC_E_CAPACITY = -7,   /* a size above a documented maximum */
    WCC_E_CFL = -8         /* a CFL number above the degree's linear stability limit */
};

/* Scheme and launch options.  wcc_default_options fills:
 *   precision = WCC_FP64, limiter = 1,
 *   alpha = 2 (Eq. 1DHighOrderWeights; Sec. 2.2 sets alpha = 2; the same
 *   value is used for P = 1, where the paper does not state it),
 *   eps = 1e-40 (Eq. 1D2ndOrderWeights), gamma = 1.4, adv_speed = 1,
 *   graph_chunk = 32 (half-steps per captured CUDA graph; 0 disables graphs),
 *   tb_depth = 1, tb_cfl_growth = 0.1 (see below), cells_per_block = 0,
 *   cuda_stream = NULL (the handle creates its own non-blocking stream).
 *
 * cells_per_block: new cells per CTA of the one-half-step kernel.  0 takes
 * the compiled default of the degree; FP32-mixed also offers 255 and 510
 * (one or two 255-cell tiles per CTA; the default is 510 for P <= 2 and 255
 * above); plain FP32 only its default; FP64 only 127.  Other values are
 * WCC_E_INVAL.  wcc_autotune picks it, with tb_depth, by timing.
 *
 * tb_depth (temporal blocking): half-steps per pass over the state in
 * device memory, 1 or 2 (0 reads as 1).  With 2 (FP32 variants only,
 * WCC_E_INVAL with WCC_FP64 or a batch), wcc_step advances the stage two
 * half-steps per launch, reading and writing the state once for both.  The
 * pair shares one dt, the CFL step of its first stage (dt = cfl dx /
 * a_max(t^n)); the second half-step's own CFL number dt a_max(t^{n+1/2}) /
 * dx is checked on the device and must not exceed min(cfl (1 +
 * tb_cfl_growth), wcc_stability_limit(P)).  A pair that would is not taken:
 * wcc_step then advances from the last stage it reached with single CFL
 * half-steps (wcc_tb_stats counts these fallbacks).  The realised dt of
 * every half-step is in the history as usual.  With tb_depth = 2, wcc_step
 * waits for its work before it returns (to check the pairs). */
typedef struct {
    int precision;
    int limiter;
    double alpha;
    double eps;
    double gamma;
    double adv_speed;
    int graph_chunk;
    int tb_depth;
    void* cuda_stream; /* cudaStream_t to run on, or NULL */
    double tb_cfl_growth;
    int cells_per_block;
    int reserved;
} wcc_options;

typedef struct wcc_ctx* wcc_handle;

void wcc_default_options(wcc_options* opt);

/* Create a solver for `system` on [domain[0], domain[1]] with N cells of
 * width dx and polynomial degree P (order P+1, Sec. 2.1): 1 <= P <= 6 in
 * every precision (WCC_E_INVAL otherwise).  The paper prints CFL numbers up to P = 3; the von Neumann
 * limits of the linear scheme (Sec. 2.3) are 0.282, 0.212 and 0.185 at
 * P = 4, 5, 6, and the CFL number must stay below them.
 * 4 <= N <= 2^31; bc is WCC_BC_PERIODIC or WCC_BC_TRANSMISSIVE.  opt may
 * be NULL.  On success *out holds the handle (free with wcc_destroy).
 * Allocates, on the current device, two stages (FP64: nv (P+1) doubles per
 * cell; FP32 variants: nv (P+2) floats), a host-layout staging buffer and
 * the device-side state (wcc_device_bytes reports the total).  Errors:
 * WCC_E_INVAL (arguments), WCC_E_CUDA (no device, stream), WCC_E_NOMEM (the
 * state does not fit, e.g. N = 2^31 at P = 6 in FP64); *out is set to NULL
 * on every error but a NULL out. */
int wcc_create(wcc_handle* out, int system, int64_t N, int P, const double domain[2], int bc,
               const wcc_options* opt);

/* Number of cells of the current stage (see the stage rules above). */
int wcc_num_cells(wcc_handle h, int64_t* ncells);

/* Load an integer stage (t = 0, parity 0) from host FP64 DOFs
 * [cell][var][k] (see layout above); count must equal cells*nv*(P+1) of an
 * integer stage.  Synchronous; also evaluates the CFL bound of the stage. */
int wcc_set_initial(wcc_handle h, const double* dofs, int64_t count);

/* Advance nsteps half-steps with dt = cfl * dx / a_max, a_max the largest
 * characteristic speed (|a|, |u| or |u| + c) over the centre point values of
 * the stage being advanced, evaluated on the device (no host round trip).
 * 0 < cfl <= wcc_stability_limit(P) (the von Neumann limit of the linear
 * scheme, Sec. 2.3); a larger cfl is WCC_E_CFL and takes no step.
 * Asynchronous on the handle's stream (with tb_depth = 2: the half-steps go
 * in pairs and the call waits for them, see wcc_options). */
int wcc_step(wcc_handle h, int64_t nsteps, double cfl);

/* Autotuner of the single-grid launch: times every compiled launch
 * configuration of the handle -- for FP32-mixed cells_per_block 255 and 510
 * with one half-step per launch, and two half-steps per launch -- on the
 * handle's own current stage at CFL number cfl (a warm-up graph, then three
 * graphs of graph_chunk half-steps each, CUDA events on the handle's
 * stream), keeps the fastest in the handle's options and reports it in
 * *cells_per_block and *tb_depth (either may be NULL).  The stage, its time
 * and step count and the dt history are restored afterwards (the launch
 * count is not).  FP64 and plain FP32 handles have one configuration each,
 * which is returned untimed.  Allocates a copy of the stage while it runs.
 * Synchronous.  Errors: WCC_E_STATE before wcc_set_initial, WCC_E_INVAL
 * (cfl), WCC_E_NOMEM, WCC_E_CUDA. */
int wcc_autotune(wcc_handle h, double cfl, int* cells_per_block, int* tb_depth);

/* Two-half-step launches (tb_depth = 2) since wcc_set_initial: *pairs (may
 * be NULL) receives the pairs taken, *fallbacks the pairs refused by the CFL
 * check and re-done as single half-steps, *nu2_max the largest CFL number a
 * taken pair's second half-step had.  Synchronises. */
int wcc_tb_stats(wcc_handle h, int64_t* pairs, int64_t* fallbacks, double* nu2_max);

/* Advance nsteps half-steps with the given half-step sizes (host array of
 * nsteps doubles, each > 0).  Asynchronous; dts is read before return. */
int wcc_step_dt(wcc_handle h, int64_t nsteps, const double* dts);

/* Advance from the current time to t_end, ending on an integer stage
 * (the reading of the paper's Table 2 runs, which do not say how t_end is
 * hit): CFL half-steps (as wcc_step) in pairs while a pair fits, then the
 * remaining time split into two equal half-steps.  Each half-step's CFL size
 * is the one the kernels will take (read from the device between steps), so
 * the decision is exact; near t_end this synchronises after every
 * half-step.  A rest below 1e-9 of a half-step counts as the rounding of the
 * summed time and is not stepped.  If the second CFL step of a pair would pass t_end, the rest of
 * the time is taken in one step.  Must start on an integer stage
 * (WCC_E_STATE otherwise); t_end before the current time is WCC_E_INVAL.
 * *nsteps_taken (may be NULL) receives the number of half-steps taken.
 * cfl as in wcc_step (WCC_E_CFL above the stability limit).
 * Synchronous; reports device-side errors. */
int wcc_step_until(wcc_handle h, double t_end, double cfl, int64_t* nsteps_taken);

/* Copy the current stage to host FP64 DOFs [cell][var][k] (count =
 * cells*nv*(P+1) of the current stage).  Synchronises the stream and
 * reports any device-side error raised since the last check. */
int wcc_get_dofs(wcc_handle h, double* dofs, int64_t count);

/* Time, number of half-steps taken and stage parity (0: integer stage,
 * 1: half stage).  Synchronises and reports device-side errors. */
int wcc_get_state(wcc_handle h, double* t, int64_t* half_steps, int* parity);

/* Half-step sizes actually used, oldest first: copies min(cap, taken)
 * values to dts and sets *n to the number taken since wcc_set_initial. */
int wcc_get_dt_history(wcc_handle h, double* dts, int64_t cap, int64_t* n);

/* Wait for all work queued on the handle; reports device-side errors. */
int wcc_synchronize(wcc_handle h);

/* Device memory footprint of the handle in bytes. */
int wcc_device_bytes(wcc_handle h, int64_t* bytes);

/* Number of kernel launches (graph nodes included) enqueued by the handle
 * since wcc_create. */
int wcc_launch_count(wcc_handle h, int64_t* launches);

/* ------------------------------------------------------------------ batches
 * Many independent problems of one conservation law, advanced together: one
 * persistent kernel launch per half-step walks the tiles of every instance
 * (cells are flattened across instances, so instances of very different N
 * share the GPU evenly).  Each instance keeps its own N, P, domain, boundary,
 * time and dt = cfl * dx_i / a_max,i (the scheme of Sec. 2 applied to each
 * problem independently).  Batches run in WCC_FP32_MIXED precision only and
 * hold at most two different degrees P.
 *
 * Host layout of a batch: the instances one after another in the user's
 * order, each as in wcc_set_initial ([cell][var][k] of u_kx, cells of its
 * current stage: N_i (periodic) or N_i + 1 / N_i (transmissive, integer /
 * half stage)).  wcc_batch_dof_count gives the total number of doubles. */
typedef struct wcc_batch_ctx* wcc_batch;

/* count instances; N[count], P[count] (1..4, at most two distinct values),
 * domains[2*count] (x_L, x_R per instance), bcs[count]; opt may be NULL but
 * opt->precision must be WCC_FP32_MIXED when given.  opt->tb_depth 2 (two
 * half-steps per launch, one dt per instance and pair, as for a single
 * problem) is taken for the degree mixes {2}, {3} and {2, 3} only; a pair is
 * refused for the whole batch when any instance's second half-step would
 * exceed its bound (opt->tb_cfl_growth, capped at the degree's linear
 * stability limit) and the batch then takes the two half-steps singly.
 * opt->cells_per_block must be 0 or 255 (the batch kernel's tile). */
int wcc_batch_create(wcc_batch* out, int system, int64_t count, const int64_t* N, const int* P,
                     const double* domains, const int* bcs, const wcc_options* opt);
int wcc_batch_dof_count(wcc_batch b, int64_t* count);
/* Load integer stages of all instances (t = 0); synchronous. */
int wcc_batch_set_initial(wcc_batch b, const double* dofs, int64_t count);
/* nsteps half-steps of every instance, each with its own CFL dt;
 * asynchronous.  cfl above the stability limit of either degree is
 * WCC_E_CFL. */
int wcc_batch_step(wcc_batch b, int64_t nsteps, double cfl);
int wcc_batch_get_dofs(wcc_batch b, double* dofs, int64_t count);
/* t[count]: the time of every instance (user order). */
int wcc_batch_get_times(wcc_batch b, double* t, int64_t count);
int wcc_batch_get_state(wcc_batch b, int64_t* half_steps, int* parity);
/* Half-step sizes of one instance (user index), as wcc_get_dt_history. */
int wcc_batch_get_dt_history(wcc_batch b, int64_t instance, double* dts, int64_t cap, int64_t* n);
/* Persistent grid of the step kernel in CTAs (0: all resident CTAs). */
int wcc_batch_set_grid(wcc_batch b, int ctas);
/* Time the candidate grids (1..max resident CTAs per SM, and one CTA per
 * tile), each with one half-step per launch and, where the degree mix has
 * the kernel (degrees {2}, {3}, {2, 3}), two; keep the fastest pair of grid
 * and pass depth, and restore the batch state.  Timed over eight half-steps
 * of this batch with this CFL number; a two-half-step candidate that had a
 * pair refused while it was timed is not taken.  *ctas (may be NULL) receives the grid;
 * wcc_batch_get_tuning reports both.  Allocates a temporary copy of the
 * current stage.  Synchronous. */
int wcc_batch_autotune(wcc_batch b, double cfl, int* ctas);
/* The launch configuration in use: *ctas the persistent grid of the step
 * kernel, *tb_depth half-steps per launch (1 or 2).  Either may be NULL. */
int wcc_batch_get_tuning(wcc_batch b, int* ctas, int* tb_depth);
/* Two-half-step launches of a batch: *pairs taken, *fallbacks refused (a
 * refused pair leaves every instance untouched and is re-done as two single
 * half-steps).  Either may be NULL.  Synchronises the batch's stream. */
int wcc_batch_tb_stats(wcc_batch b, int64_t* pairs, int64_t* fallbacks);
int wcc_batch_synchronize(wcc_batch b);
int wcc_batch_launch_count(wcc_batch b, int64_t* launches);
int wcc_batch_device_bytes(wcc_batch b, int64_t* bytes);
const char* wcc_batch_last_error(wcc_batch b);
void wcc_batch_destroy(wcc_batch b);

/* Linear stability limit of degree P (1..6): the largest CFL number nu with
 * which one half-step of linear advection (limiter off) keeps every Fourier
 * mode bounded -- every eigenvalue of the half-step amplification matrix
 * G(theta) = M_L e^{-i theta/2} + M_R e^{i theta/2} in the closed unit disk
 * (Sec. 2.3, Eqs. 1DSchemeMatrixForm, 1DFourierAnalysis,
 * LinearStabilityCondition), found by bisection over 2047 values of theta.
 * Host code, no device needed; computed on the first call for each P (about
 * 0.1-1 s) and kept.  The paper's Table 1 prints 0.5, 0.384 and 0.304 for
 * P = 1, 2, 3; this scan gives 0.5, 0.384 and 0.289 (at 0.304 the radius
 * exceeds 1 by about 1e-4).  Errors: WCC_E_INVAL (P out of range, NULL). */
int wcc_stability_limit(int P, double* nu);

/* Default CFL number (half-step nu = a_max dt / dx) of degree P (1..6):
 * the values the paper's numerical tests use for P = 1, 2, 3 (0.4, 0.3,
 * 0.25; Sec. 5), and for P >= 4, where the paper gives none, 0.8 of
 * wcc_stability_limit(P) rounded down to two digits (0.22, 0.16, 0.14 for
 * P = 4, 5, 6).  Errors: WCC_E_INVAL. */
int wcc_default_cfl(int P, double* cfl);

/* Measured fused-multiply-add throughput of the current device in TFLOP/s
 * (FP64 for WCC_FP64, FP32 for WCC_FP32_MIXED): a grid of 8 CTAs per SM,
 * 8 independent FMA chains per thread, timed with CUDA events (~40 ms).
 * The roofline denominator of ALU-bound kernels; the paper has no
 * counterpart. */
int wcc_measure_fp_peak(int precision, double* tflops);

/* Largest nsteps accepted by wcc_advance_static. */
#define WCC_STATIC_MAX_HALFSTEPS 4096

/* Allocation-free stepping (the paper has no counterpart; this is a service
 * for callers that cannot allocate device memory when they step -- e.g. a
 * host application whose own allocator owns the device memory pool, or a
 * code path that must avoid the device-wide synchronisation a cudaMalloc /
 * cudaFree may cause).  It runs the FP64 half-step kernels of wcc_step
 * nsteps times with dt = cfl * dx / a_max from the device, on two stage
 * buffers the caller owns, and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Arguments: system, P (1..6), bc, N (4..2^31), domain as in wcc_create; opt may be
 * NULL (opt->precision must be WCC_FP64; opt->cuda_stream is the stream,
 * NULL = legacy default stream).  parity is the stage parity of the input.
 * cfl as in wcc_step (WCC_E_CFL above the degree's stability limit).
 * stage_a (input) and stage_b are device buffers of nv*(P+1) FP64 planes,
 * plane (v, k) at offset (v*(P+1) + k) * pitch elements, holding the Taylor
 * coefficients e_k = u_kx / k! of cell i at index i; pitch >= N + 1, both
 * 8-byte aligned and distinct.  The stages alternate a -> b -> a ...: after
 * the call the final stage is in stage_a if nsteps is even, else in stage_b.
 * dts_out (host, may be NULL) receives the nsteps half-step sizes.
 *
 * Scratch: a fixed array of about 33 KB in the library's device image (the
 * CFL accumulators, counters, error bits and a dt history of
 * WCC_STATIC_MAX_HALFSTEPS entries); every GPU that loads the library holds
 * it until the process exits.  nsteps > WCC_STATIC_MAX_HALFSTEPS returns
 * WCC_E_CAPACITY.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  The lookup is repeated when the device's
 * context has changed since (e.g. after a cudaDeviceReset, which reloads the
 * library's device code), so the first call after a reset must also come
 * before any capture.  All calls share the array and each call
 * clears its state first, so calls that overlap on the GPU (other streams,
 * other host threads) race and must not be made.
 *
 * Synchronous: returns after the stream has finished, with WCC_OK or
 * WCC_E_INVAL / WCC_E_CAPACITY / WCC_E_CUDA / WCC_E_NONFINITE /
 * WCC_E_POSITIVITY (no message is kept for this call). */
int wcc_advance_static(int system, int P, int bc, int64_t N, const double domain[2], const wcc_options* opt,
                       int parity, double* stage_a, double* stage_b, int64_t pitch, int64_t nsteps, double cfl,
                       double* dts_out);

const char* wcc_last_error(wcc_handle h);
void wcc_destroy(wcc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* WCC_H */
