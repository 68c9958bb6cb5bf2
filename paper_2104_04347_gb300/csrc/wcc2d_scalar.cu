// 2D scalar half-step kernels (linear advection, Burgers; FP64 and FP32,
// P = 1..3), the stage CFL-rate kernels, and the dispatch of every 2D launch.
#include "wcc2d_kernels.cuh"

namespace wcc2d {

cudaError_t launch_halfstep2d_euler_f64(int P, const Step2D& a, cudaStream_t stream);
cudaError_t launch_halfstep2d_euler_f32(int P, const Step2D& a, cudaStream_t stream);

cudaError_t launch_halfstep2d(int system, int P, bool fp32, const Step2D& a, cudaStream_t stream) {
    switch (system) {
        case ADVECTION:
            return fp32 ? launch_halfstep2d_sys<ADVECTION, float>(P, a, stream)
                        : launch_halfstep2d_sys<ADVECTION, double>(P, a, stream);
        case BURGERS:
            return fp32 ? launch_halfstep2d_sys<BURGERS, float>(P, a, stream)
                        : launch_halfstep2d_sys<BURGERS, double>(P, a, stream);
        case EULER:
            return fp32 ? launch_halfstep2d_euler_f32(P, a, stream) : launch_halfstep2d_euler_f64(P, a, stream);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stage_rate2d(int system, bool fp32, const void* planes, long long pitch, long long plane, int nx,
                                int ny, int nq_, const Law2D& law, double dx, double dy, DevState2D* st,
                                cudaStream_t stream) {
    switch (system) {
        case ADVECTION:
            return launch_stage_rate2d_sys<ADVECTION>(fp32, planes, pitch, plane, nx, ny, nq_, law, dx, dy, st, stream);
        case BURGERS:
            return launch_stage_rate2d_sys<BURGERS>(fp32, planes, pitch, plane, nx, ny, nq_, law, dx, dy, st, stream);
        case EULER:
            return launch_stage_rate2d_sys<EULER>(fp32, planes, pitch, plane, nx, ny, nq_, law, dx, dy, st, stream);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace wcc2d
