/*
 * wcc2d.h -- C ABI of the GB300 (sm_103a) implementation of the 2D weighted
 * compact central (WCC) scheme of arXiv 2104.04347 (Sec. 3, Sec. 4,
 * Appendix B) for u_t + f(u)_x + g(u)_y = 0 (Eq. 2DHCL) with
 *   f = ax u, g = ay u (linear advection), f = g = u^2/2 (Burgers), or the
 *   2D Euler equations U = (rho, rho u, rho v, rho e) (Eq. 2DHCLSystem,
 *   Sec. 5.3), limited in rotated characteristic variables (Sec. 4).
 *
 * Conventions follow wcc.h: every function returns WCC_OK (0) or a negative
 * WCC_E_* code (declared there), the message of the last failure is
 * returned by wcc2d_last_error(handle) (wcc2d_last_error(NULL) for
 * wcc2d_create), and there is no CPU fallback.
 *
 * Mesh and layout (Sec. 3.1, Fig. 2DMesh):
 *   - dx = (x_E - x_S)/nx, dy = (y_E - y_S)/ny.  Integer stages hold cells
 *     centred on (x_S + i dx, y_S + j dy), half stages cells centred on
 *     (x_S + (i + 1/2) dx, y_S + (j + 1/2) dy).  Periodic: nx x ny cells per
 *     stage.  Transmissive: (nx+1) x (ny+1) cells on integer stages and
 *     nx x ny on half stages; a ghost parent is a copy of the nearest cell
 *     along each axis.
 *   - Host DOF arrays are FP64 [j][i][var][q] (row j along y, column i along
 *     x), holding the scaled derivatives u_{kx,ly} = dx^k dy^l d^k_x d^l_y u
 *     at the cell centre (Eq. 2DPolynomial_Space) for k + l <= P, at position
 *     q = (k+l)(k+l+1)/2 + l; nq = (P+1)(P+2)/2 per variable, nv = 1 or 4.
 *   - Time steps are HALF steps (t^{n+1/2} - t^n).  The CFL rule is
 *     dt = cfl / max over the cells of the stage being advanced of
 *     (s_x/dx + s_y/dy), s the characteristic speed along each axis
 *     (|ax|, |ay|; |u|; |u| + c, |v| + c) at the cell centre; the paper does
 *     not state a 2D rule, and this one reproduces its Table 3.
 *   - The device layout is private: planes [var][q][row][col] of FP64
 *     (WCC_FP64) or FP32 values; WCC_FP32_MIXED keeps the cell average (as
 *     a float-float pair) in place of the point value.
 *
 * Ownership and threads: as in wcc.h.  The handle owns its device memory;
 * caller buffers are borrowed for the call only; one call at a time per
 * handle, from any host thread.
 */
#ifndef WCC2D_H
#define WCC2D_H

#include <stdint.h>

#include "wcc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Options.  wcc2d_default_options fills: precision = WCC_FP64, limiter = 1,
 * alpha = 2, eps = 1e-40 (Eq. 2D2ndOrderWeights), gamma = 1.4, ax = ay = 1,
 * rows_per_cta = 16 (new rows one CTA marches through), cuda_stream = NULL
 * (the handle creates its own non-blocking stream).  precision is WCC_FP64,
 * WCC_FP32 (every value and operation in float) or WCC_FP32_MIXED (float
 * arithmetic, with the cell average, the leading flux terms and the vertex
 * point values in float-float, so that the averages keep about 48 bits). */
typedef struct {
    int precision;
    int limiter;
    double alpha;
    double eps;
    double gamma;
    double ax, ay;
    int rows_per_cta;
    int reserved;
    void* cuda_stream;
} wcc2d_options;

typedef struct wcc2d_ctx* wcc2d_handle;

void wcc2d_default_options(wcc2d_options* opt);

/* Create a solver for `system` (WCC_ADVECTION, WCC_BURGERS or WCC_EULER) on
 * [domain[0], domain[1]] x [domain[2], domain[3]] with nx x ny cells and
 * degree 1 <= P <= 3 (order P + 1).  nx, ny >= 4 and at most 2^15 each;
 * bc is WCC_BC_PERIODIC or WCC_BC_TRANSMISSIVE.  opt may be NULL.
 * Allocates two stages, a host-layout staging buffer and the device-side
 * state on the current device (wcc2d_device_bytes reports the total); it
 * changes no context-wide setting.  Errors: WCC_E_INVAL, WCC_E_CAPACITY (nx
 * or ny above 2^15), WCC_E_NOMEM, WCC_E_CUDA (no device or stream); *out is
 * set to NULL on every error but a NULL out. */
int wcc2d_create(wcc2d_handle* out, int system, int64_t nx, int64_t ny, int P, const double domain[4], int bc,
                 const wcc2d_options* opt);

/* Cells along x and y of the current stage. */
int wcc2d_stage_dims(wcc2d_handle h, int64_t* nx, int64_t* ny);

/* Load an integer stage (t = 0, parity 0) from host FP64 DOFs (layout
 * above); count = cells * nv * nq of an integer stage.  Synchronous; also
 * evaluates the CFL rate of the stage (reports WCC_E_POSITIVITY /
 * WCC_E_NONFINITE for non-physical or non-finite centre values). */
int wcc2d_set_initial(wcc2d_handle h, const double* dofs, int64_t count);

/* nsteps CFL half-steps (rule above; cfl > 0), asynchronous. */
int wcc2d_step(wcc2d_handle h, int64_t nsteps, double cfl);

/* nsteps half-steps of the given sizes (each > 0), asynchronous. */
int wcc2d_step_dt(wcc2d_handle h, int64_t nsteps, const double* dts);

/* Advance to t_end, ending on an integer stage: CFL half-steps in pairs
 * while a pair fits, then the rest in two equal half-steps (if the second
 * CFL step of a pair would pass t_end, the rest in one step); the CFL size
 * of each half-step is read from the device.  Starts on an integer stage
 * (WCC_E_STATE otherwise); t_end before the current time is WCC_E_INVAL.
 * Synchronous; *nsteps_taken (may be NULL) receives the half-steps taken. */
int wcc2d_step_until(wcc2d_handle h, double t_end, double cfl, int64_t* nsteps_taken);

/* Copy the current stage to host FP64 DOFs; count = cells * nv * nq of the
 * current stage.  Synchronises and reports device-side errors. */
int wcc2d_get_dofs(wcc2d_handle h, double* dofs, int64_t count);

/* Time, half-steps taken, stage parity.  Synchronises, reports errors. */
int wcc2d_get_state(wcc2d_handle h, double* t, int64_t* steps, int* parity);

/* Half-step sizes taken since the last wcc2d_set_initial: *n (may be NULL)
 * receives how many were taken; the first min(n, cap) are copied to dts. */
int wcc2d_get_dt_history(wcc2d_handle h, double* dts, int64_t cap, int64_t* n);

/* Wait for queued work; reports device-side errors. */
int wcc2d_synchronize(wcc2d_handle h);

/* Autotuner of the strip height: times rows_per_cta = 8 .. 24 (13
 * candidates; the count of CTAs, and so how full the last wave of resident
 * CTAs is, changes with it) on the handle's own current stage at CFL number
 * cfl, one warm-up and four timed half-steps each (CUDA events on the
 * handle's stream), keeps the fastest in the handle's options and reports it
 * in *rows_per_cta (may be NULL).  The stage, its time and step count and the
 * dt history are restored afterwards (the launch count is not); the results
 * of later half-steps do not depend on the strip height.  Allocates a copy of
 * the stage while it runs.  Synchronous.  Errors: WCC_E_STATE before
 * wcc2d_set_initial, WCC_E_INVAL (cfl), WCC_E_NOMEM, WCC_E_CUDA, and the
 * device-side errors of the timed half-steps (the state is restored). */
int wcc2d_autotune(wcc2d_handle h, double cfl, int* rows_per_cta);

/* Kernel launches issued by this handle since creation. */
int wcc2d_launch_count(wcc2d_handle h, int64_t* n);

/* Device bytes owned by the handle. */
int wcc2d_device_bytes(wcc2d_handle h, int64_t* bytes);

const char* wcc2d_last_error(wcc2d_handle h);

/* Release the handle and its device memory (NULL is a no-op). */
int wcc2d_destroy(wcc2d_handle h);

#ifdef __cplusplus
}
#endif

#endif /* WCC2D_H */
