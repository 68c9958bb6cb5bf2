// 2D FP32-mixed half-step kernels (advection, Burgers, Euler; P = 1..3), the
// stage CFL rate and the layout conversions of the FP32-mixed storage.
#include "wcc2d_kernels.cuh"

namespace wcc2d {

namespace {
template <int SYS>
cudaError_t launch_mx_sys(int P, const Step2D& a, cudaStream_t stream) {
    switch (P) {
        case 1: return launch_halfstep2d_mx_t<SYS, 1>(a, stream);
        case 2: return launch_halfstep2d_mx_t<SYS, 2>(a, stream);
        case 3: return launch_halfstep2d_mx_t<SYS, 3>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int SYS, int P>
cudaError_t rate_mx_t(const float* planes, long long pitch, long long plane, int nx, int ny, const Law2D& law,
                      double dx, double dy, DevState2D* st, cudaStream_t stream) {
    const long long n = (long long)nx * ny;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 8);
    stage_rate2d_mx<SYS, P><<<grid, 256, 0, stream>>>(planes, pitch, plane, nx, ny, law, dx, dy, st);
    return cudaGetLastError();
}

template <int SYS>
cudaError_t rate_mx_sys(int P, const float* planes, long long pitch, long long plane, int nx, int ny,
                        const Law2D& law, double dx, double dy, DevState2D* st, cudaStream_t stream) {
    switch (P) {
        case 1: return rate_mx_t<SYS, 1>(planes, pitch, plane, nx, ny, law, dx, dy, st, stream);
        case 2: return rate_mx_t<SYS, 2>(planes, pitch, plane, nx, ny, law, dx, dy, st, stream);
        case 3: return rate_mx_t<SYS, 3>(planes, pitch, plane, nx, ny, law, dx, dy, st, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_halfstep2d_mx(int system, int P, const Step2D& a, cudaStream_t stream) {
    switch (system) {
        case ADVECTION: return launch_mx_sys<ADVECTION>(P, a, stream);
        case BURGERS: return launch_mx_sys<BURGERS>(P, a, stream);
        case EULER: return launch_mx_sys<EULER>(P, a, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stage_rate2d_mx(int system, int P, const float* planes, long long pitch, long long plane, int nx,
                                   int ny, const Law2D& law, double dx, double dy, DevState2D* st, cudaStream_t stream) {
    switch (system) {
        case ADVECTION: return rate_mx_sys<ADVECTION>(P, planes, pitch, plane, nx, ny, law, dx, dy, st, stream);
        case BURGERS: return rate_mx_sys<BURGERS>(P, planes, pitch, plane, nx, ny, law, dx, dy, st, stream);
        case EULER: return rate_mx_sys<EULER>(P, planes, pitch, plane, nx, ny, law, dx, dy, st, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_convert2d_mx(int P, bool to_planes, double* aos, float* planes, int nx, int ny, int nv,
                                long long pitch, long long plane, cudaStream_t stream) {
    const long long n = (long long)nx * ny;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    switch (P) {
        case 1:
            if (to_planes) aos_to_planes2d_mx<1><<<grid, 256, 0, stream>>>(aos, planes, nx, ny, nv, pitch, plane);
            else planes_to_aos2d_mx<1><<<grid, 256, 0, stream>>>(planes, aos, nx, ny, nv, pitch, plane);
            break;
        case 2:
            if (to_planes) aos_to_planes2d_mx<2><<<grid, 256, 0, stream>>>(aos, planes, nx, ny, nv, pitch, plane);
            else planes_to_aos2d_mx<2><<<grid, 256, 0, stream>>>(planes, aos, nx, ny, nv, pitch, plane);
            break;
        case 3:
            if (to_planes) aos_to_planes2d_mx<3><<<grid, 256, 0, stream>>>(aos, planes, nx, ny, nv, pitch, plane);
            else planes_to_aos2d_mx<3><<<grid, 256, 0, stream>>>(planes, aos, nx, ny, nv, pitch, plane);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace wcc2d
