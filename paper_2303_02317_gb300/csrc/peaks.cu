// peaks.cu -- measured arithmetic peaks of this GPU (a diagnostic beside the
// pricer, not part of the paper's method).
//
// The pricer's transforms and base cases run on the FP32 pipe (doubled FP32
// and FP32 hi/lo values) and a few steps on the FP64 pipe; their roofline
// fraction needs the rate those pipes reach on this part, measured rather
// than derived from unit counts.  fma_peak_kernel keeps eight independent
// FMA chains per thread (enough to cover the pipe latency) in every lane of
// a grid of 8 CTAs x 256 threads per SM and runs them for a fixed count; the
// result is stored so that the compiler keeps the work.

#include <cuda_runtime.h>

#include "american.h"
#include "internal.h"

namespace aop {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(int iters, T a, T b, T *out)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 16; r++) {
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == (T)12345.678) out[blockIdx.x] = s;   // never true for the inputs used; keeps the chains live
}

template <class T>
cudaError_t time_peak(int device, int iters, double *flops_per_s) {
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const int grid = sms * kCtasPerSm;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    T *out = nullptr;
    float best = -1.f;
    // out is never written (see the kernel): a null pointer is not dereferenced
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, 0);
        fma_peak_kernel<T><<<grid, kThreads>>>(iters, (T)0.999999, (T)1e-7, out);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best < 0.f || ms < best)) best = ms;   // rep 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double fmas = (double)grid * kThreads * (double)iters * 16.0 * kChains;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace
}  // namespace aop

extern "C" aop_status aop_measure_fma_peak(int device, int bits, double *flops_per_s)
{
    using namespace aop;
    if (!flops_per_s || (bits != 32 && bits != 64)) return AOP_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return AOP_ECUDA; }
    // about 0.1 s a run at either pipe's rate on a GB300 (80 TFLOP/s FP32
    // nominal, 1.25 FP64)
    const cudaError_t e = (bits == 32) ? time_peak<float>(device, 100000, flops_per_s)
                                       : time_peak<double>(device, 1500, flops_per_s);
    if (e != cudaSuccess) { cudaGetLastError(); return AOP_ECUDA; }
    return AOP_OK;
}
