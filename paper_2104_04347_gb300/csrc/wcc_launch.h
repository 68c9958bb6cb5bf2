// wcc_launch.h -- host-side entry points of the per-system kernel
// translation units (wcc_kernels_<system>.cu).
#pragma once

#include <cuda_runtime.h>

#include "wcc_scheme.cuh"

namespace wcc {

// One fused half-step over a whole stage: grid = ceil(n_new / kTile) CTAs.
template <int SYS>
cudaError_t launch_halfstep(int P, int precision, const StepArgs& args, cudaStream_t stream);

// Largest characteristic speed of the stage whose centre point values start
// at u0planes (variable v at u0planes + v * var_stride); result in
// st->amax_bits[slot], which must be zero beforehand.
template <int SYS>
cudaError_t launch_stage_speed(const double* u0planes, long long var_stride, long long n,
                               const StepArgs& args, int slot, cudaStream_t stream);

// Same for an FP32-mixed stage (planes [v][ubar hi, ubar lo, e_1..e_P][cell]).
template <int SYS>
cudaError_t launch_stage_speed_mixed(int P, const float* planes, long long pitch, long long n,
                                     const StepArgs& args, int slot, cudaStream_t stream);

inline unsigned halfstep_grid(long long n_new) { return (unsigned)((n_new + kTile - 1) / kTile); }

}  // namespace wcc
