// wcc_launch.h -- host-side entry points of the per-system kernel
// translation units (wcc_kernels_<system>.cu).
#pragma once

#include <cuda_runtime.h>

#include "wcc_scheme.cuh"

namespace wcc {

// One fused half-step over a whole stage: grid = ceil(n_new / kTile) CTAs.
template <int SYS>
cudaError_t launch_halfstep(int P, int precision, const StepArgs& args, cudaStream_t stream);
// its FP64 and FP32-variant parts (compiled in separate translation units)
template <int SYS>
cudaError_t launch_halfstep_fp64(int P, const StepArgs& args, cudaStream_t stream);
template <int SYS>
cudaError_t launch_halfstep_mixed(int P, int precision, const StepArgs& args, cudaStream_t stream);
// the FP32-variant kernels at P = 5, 6 (one- and two-half-step)
template <int SYS>
cudaError_t launch_halfstep_mixed_hi(int P, int precision, const StepArgs& args, cudaStream_t stream);
template <int SYS>
cudaError_t launch_halfstep_pair_hi(int P, int precision, const StepArgs& args, cudaStream_t stream);

// Two half-steps in one launch (FP32 variants, P <= 4; halfstep_mixed2_tb2):
// args.in32 -> args.out32 with args.n_mid cells in between;
// grid = ceil(n_new / kTileTB) CTAs.
template <int SYS>
cudaError_t launch_halfstep_pair(int P, int precision, const StepArgs& args, cudaStream_t stream);

// Largest characteristic speed of the stage whose centre point values start
// at u0planes (variable v at u0planes + v * var_stride); result in
// st->amax_bits[slot], which must be zero beforehand.
template <int SYS>
cudaError_t launch_stage_speed(const double* u0planes, long long var_stride, long long n,
                               const StepArgs& args, int slot, cudaStream_t stream);

// Set-up of an FP32-mixed stage (planes [v][ubar hi, ubar lo, e_1..e_P][cell],
// plane pitch `pitch`) from n cells of host-layout DOFs already in device
// memory (aos), and its largest characteristic speed into st->amax_bits[slot]
// (zero beforehand), in one pass.  keep_lo = 0 stores the plain FP32 average.
template <int SYS>
cudaError_t launch_load_stage_mixed(int P, const double* aos, long long n, long long pitch, float* planes,
                                    int keep_lo, const StepArgs& args, int slot, cudaStream_t stream);

struct BatchArgs;
enum { BATCH_STEP = 0, BATCH_SPEED = 1, BATCH_CONVERT = 2, BATCH_PAIR = 3 };

// Batched launches (wcc_batch.cuh) for groups of degree PA <= PB: one
// half-step (BATCH_STEP), two half-steps (BATCH_PAIR), the stage bound after
// loading (BATCH_SPEED), or the layout conversion (BATCH_CONVERT,
// to_planes = 1: host layout -> planes).
template <int SYS>
cudaError_t launch_batch(int PA, int PB, int kind, const BatchArgs& b, double* aos, int to_planes, unsigned grid,
                         cudaStream_t stream);

// The batched two-half-step kernel (degree mixes (2, 2), (3, 3) and (2, 3);
// cudaErrorInvalidValue for the others).
template <int SYS>
cudaError_t launch_batch_pair(int PA, int PB, const BatchArgs& b, unsigned grid, cudaStream_t stream);

// Resident CTAs per SM of the batched half-step kernel.
template <int SYS>
int batch_blocks_per_sm(int PA, int PB);

// Makes `device` current for the calling host thread for the scope of one
// library call and restores the thread's previous device afterwards: a
// handle may be used from any host thread, and the CUDA runtime's current
// device is per thread.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int device) {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != device && cudaSetDevice(device) == cudaSuccess) prev = cur;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

inline unsigned halfstep_grid(long long n_new) { return (unsigned)((n_new + kTile - 1) / kTile); }

}  // namespace wcc
