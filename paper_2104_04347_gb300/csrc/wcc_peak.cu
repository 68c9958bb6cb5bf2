// wcc_peak.cu -- FMA-chain throughput microbenchmark: the FP64 / FP32 pipe
// peaks that serve as the roofline denominators of ALU-bound kernels.
#include <cuda_runtime.h>

#include "../../include/wcc.h"

namespace {

// Eight independent FMA chains per thread hide the pipeline latency; the
// multiplier is just below one and the addend small, so the values neither
// overflow nor become subnormal.  The final sum is stored so that nothing is
// optimised away.
template <class T>
__global__ void __launch_bounds__(256) fma_chains(T* sink, long long iters, T b, T c) {
    T a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == (T)-1) sink[threadIdx.x] = s;  // practically never true; keeps the chains live
}

template <class T>
int measure(double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WCC_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WCC_E_CUDA;
    T* sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(T)) != cudaSuccess) return WCC_E_NOMEM;
    const unsigned grid = (unsigned)sms * 8u;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    long long iters = 256;
    float ms = 0.f;
    int rc = WCC_OK;
    for (int round = 0; round < 12; ++round) {
        cudaEventRecord(e0);
        fma_chains<T><<<grid, 256>>>(sink, iters, (T)0.9999999, (T)1e-7);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = WCC_E_CUDA;
            break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 40.f) break;
        iters *= 2;
    }
    if (rc == WCC_OK) {
        const double flops = 2.0 * 8.0 * (double)iters * (double)grid * 256.0;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

}  // namespace

extern "C" int wcc_measure_fp_peak(int precision, double* tflops) {
    if (!tflops) return WCC_E_INVAL;
    if (precision == WCC_FP64) return measure<double>(tflops);
    if (precision == WCC_FP32_MIXED) return measure<float>(tflops);
    return WCC_E_INVAL;
}
