// setup.cu -- per-option parameter setup (hot-path row a1) and the FFT twiddle
// tables shared by every convolution.
#include <algorithm>
#include "common.cuh"
#include "internal.h"

namespace aop {

namespace {

__global__ void params_kernel(int64_t n, const aop_request *reqs, Params *params,
                              int32_t *status, unsigned long long *tmax)
{
    unsigned long long local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const aop_request q = reqs[i];
        Params P = make_params(q);
        params[i] = P;
        if (status) status[i] = P.status;
        if (P.status == AOP_OK) local = max(local, (unsigned long long)P.T);
    }
    if (tmax) {
        for (int off = 16; off > 0; off >>= 1)
            local = max(local, __shfl_down_sync(0xffffffffu, local, off));
        if ((threadIdx.x & 31) == 0) atomicMax(tmax, local);
    }
}

// Twiddle tables, one level per transform length: entry 2^(L-1) + k holds
// e^{-2 pi i k / 2^L} for k < 2^(L-1), L = 1 .. log2n (entry 0 unused).  A
// stage of half-size 2^(L-1) reads a contiguous run, so the short transforms
// touch only the first few KB of the table.  tw64 holds (cos, sin) in FP64;
// tw32 holds (cos hi, sin hi, cos lo, sin lo), the lo parts being the FP64
// residuals of the FP32 hi parts, so hi + lo carries ~48 bits.
__global__ void twiddle_kernel(int log2n, float4 *tw32, double2 *tw64)
{
    const int64_t n = (int64_t)1 << log2n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0, c = 1.0;
        if (idx > 0) {
            const int L = 64 - __clzll((unsigned long long)idx);       // 2^(L-1) <= idx < 2^L
            const int64_t half = (int64_t)1 << (L - 1);
            // angle = -2 pi k / 2^L = -pi * (k / 2^(L-1)); sincospi takes the multiple of pi
            sincospi(-(double)(idx - half) / (double)half, &s, &c);
        }
        if (tw64) tw64[idx] = make_double2(c, s);
        if (tw32) {
            float ch = (float)c, sh = (float)s;
            float cl = (float)(c - (double)ch), sl = (float)(s - (double)sh);
            tw32[idx] = make_float4(ch, sh, cl, sl);
        }
    }
}

// One block per option (grid-stride over options); the rows of a mirrored
// option are independent.
__global__ void mirror_boundary_kernel(int64_t n, const Params *params, int32_t *bnd,
                                       const int64_t *bnd_off)
{
    for (int64_t o = blockIdx.x; o < n; o += gridDim.x) {
        const Params &P = params[o];
        if (!P.mirror || P.status != AOP_OK) continue;
        int32_t *b = bnd + bnd_off[o];
        for (int64_t i = threadIdx.x; i <= P.T; i += blockDim.x)
            b[i] = (int32_t)((int64_t)P.D * i - 1 - b[i]);
    }
}

__global__ void fill_i32_kernel(int32_t *p, int64_t n, int32_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

cudaError_t launch_params(int64_t n, const aop_request *d_reqs, Params *d_params,
                          int32_t *d_status, int64_t *d_tmax, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    params_kernel<<<blocks, 256, 0, s>>>(n, d_reqs, d_params, d_status,
                                         (unsigned long long *)d_tmax);
    return cudaGetLastError();
}

cudaError_t launch_mirror_boundaries(int64_t n, const Params *d_params, int32_t *d_bnd,
                                     const int64_t *d_bnd_off, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>(n, 1024);
    mirror_boundary_kernel<<<blocks, 256, 0, s>>>(n, d_params, d_bnd, d_bnd_off);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(int log2n, void *d_tw32, void *d_tw64, cudaStream_t s)
{
    const int64_t n = (int64_t)1 << log2n;      // entries per table
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    twiddle_kernel<<<blocks, 256, 0, s>>>(log2n, (float4 *)d_tw32, (double2 *)d_tw64);
    return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    fill_i32_kernel<<<blocks, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

}  // namespace aop
