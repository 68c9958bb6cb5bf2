// 2D Euler half-step kernels in FP64 (P = 1..3).
#include "wcc2d_kernels.cuh"

namespace wcc2d {
cudaError_t launch_halfstep2d_euler_f64(int P, const Step2D& a, cudaStream_t stream) {
    return launch_halfstep2d_sys<EULER, double>(P, a, stream);
}
}  // namespace wcc2d
