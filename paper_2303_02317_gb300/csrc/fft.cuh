// fft.cuh -- FFT convolution engine for the linear advance of a row segment
// (the FFT-based linear-stencil step the trapezoid algorithm calls, Sec. 3.3
// "Solving a Trapezoid", and the periodic-grid method it cites).
//
// A linear advance of h steps is a correlation of the row segment with the
// h-fold power of the stencil.  With the forward transform X[m] = sum x[n]
// e^{-2 pi i m n / N}, the correlation out[x] = sum_o c_o in[x + o] becomes
// OUT[m] = IN[m] * s(theta_m)^h,  s(theta) = sum_o w_o e^{i theta o},
// theta_m = 2 pi m / N.  The transform is a decimation-in-frequency pass
// (natural order in, bit-reversed out); the pointwise product indexes the
// kernel power by the bit-reversed bin, and the inverse is a
// decimation-in-time pass (bit-reversed in, natural out), so no reordering pass
// is ever made.  Outputs whose correlation window wraps around are discarded.
//
// Two arithmetic modes:
//   MODE 0: FP64 complex values (double2), FP64 twiddles.
//   MODE 1: FP32 complex values (float2) carrying hi + i*lo of the FP64 input
//           (hi = fl32(x), lo = fl32(x - hi)); because the stencil power is
//           real, the real part of the result is conv(hi) and the imaginary
//           part conv(lo).  Twiddles and the kernel power are FP32 hi/lo pairs
//           applied with a compensated product.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace aop {
namespace fft {

template <int MODE> struct Cx;
template <> struct Cx<0> { using V = double2; using Tw = double2; using Sp = double2; };
template <> struct Cx<1> { using V = float2;  using Tw = float4;  using Sp = float4; };

// ------------------------------------------------------------- complex ops
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i and by +i
__device__ __forceinline__ double2 cmul_mi(double2 a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ double2 cmul_pi(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 cmul_pi(float2 a) { return make_float2(-a.y, a.x); }

// v * w (CONJ: v * conj(w))
template <bool CONJ>
__device__ __forceinline__ double2 twmul(double2 v, double2 w) {
    double s = CONJ ? -w.y : w.y;
    return make_double2(fma(v.x, w.x, -v.y * s), fma(v.x, s, v.y * w.x));
}
// compensated: w = (hi.x, hi.y, lo.x, lo.y); v * (hi + lo) with the small
// product formed first so that it is not lost.
template <bool CONJ>
__device__ __forceinline__ float2 twmul(float2 v, float4 w) {
    float sh = CONJ ? -w.y : w.y;
    float sl = CONJ ? -w.w : w.w;
    float re_lo = fmaf(v.x, w.z, -v.y * sl);
    float im_lo = fmaf(v.x, sl, v.y * w.z);
    float re = fmaf(v.x, w.x, fmaf(-v.y, sh, re_lo));
    float im = fmaf(v.x, sh, fmaf(v.y, w.x, im_lo));
    return make_float2(re, im);
}

// Twiddle e^{-2 pi i k / 2^lg} for 0 <= k < 2^(lg-1) from the table of the
// largest transform 2^tw_log2 (entries k' < 2^(tw_log2-1)).
template <int MODE>
__device__ __forceinline__ typename Cx<MODE>::Tw tw_get(const typename Cx<MODE>::Tw *tab, int tw_log2,
                                                       int64_t k, int lg) {
    return __ldg(&tab[k << (tw_log2 - lg)]);
}

__device__ __forceinline__ uint32_t brev_n(uint32_t p, int lgN) {
    return lgN == 0 ? 0u : (__brev(p) >> (32 - lgN));
}

// --------------------------------------------------- in-place stage kernels
// All threads of the block (nthr = blockDim.x) cooperate; x is N values in
// shared or global memory.  Caller synchronises between calls.

// one radix-2 DIF stage of half-size M
template <int MODE, class V>
__device__ __forceinline__ void dif2(V *x, int64_t N, int64_t M, const typename Cx<MODE>::Tw *tw,
                                     int tw_log2, int lgM2) {
    for (int64_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
        int64_t k = t & (M - 1);
        int64_t j = ((t - k) << 1) + k;
        V u = x[j], v = x[j + M];
        x[j] = cadd(u, v);
        x[j + M] = twmul<false>(csub(u, v), tw_get<MODE>(tw, tw_log2, k, lgM2));
    }
}
// one radix-2 DIT (inverse) stage of half-size M
template <int MODE, class V>
__device__ __forceinline__ void dit2(V *x, int64_t N, int64_t M, const typename Cx<MODE>::Tw *tw,
                                     int tw_log2, int lgM2) {
    for (int64_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
        int64_t k = t & (M - 1);
        int64_t j = ((t - k) << 1) + k;
        V u = x[j];
        V v = twmul<true>(x[j + M], tw_get<MODE>(tw, tw_log2, k, lgM2));
        x[j] = cadd(u, v);
        x[j + M] = csub(u, v);
    }
}
// two DIF stages (half-sizes M and M/2) as one radix-4 pass, M >= 2
template <int MODE, class V>
__device__ __forceinline__ void dif4(V *x, int64_t N, int64_t M, const typename Cx<MODE>::Tw *tw,
                                     int tw_log2, int lgM2) {
    const int64_t h = M >> 1;
    for (int64_t t = threadIdx.x; t < N / 4; t += blockDim.x) {
        int64_t k = t & (h - 1);
        int64_t j = ((t - k) << 2) + k;
        V a0 = x[j], a1 = x[j + h], a2 = x[j + M], a3 = x[j + M + h];
        auto w1 = tw_get<MODE>(tw, tw_log2, k, lgM2);       // e^{-2 pi i k/(2M)}
        auto w2 = tw_get<MODE>(tw, tw_log2, k, lgM2 - 1);   // e^{-2 pi i k/M}
        V b0 = cadd(a0, a2), b2 = twmul<false>(csub(a0, a2), w1);
        V b1 = cadd(a1, a3), b3 = cmul_mi(twmul<false>(csub(a1, a3), w1));
        x[j] = cadd(b0, b1);
        x[j + h] = twmul<false>(csub(b0, b1), w2);
        x[j + M] = cadd(b2, b3);
        x[j + M + h] = twmul<false>(csub(b2, b3), w2);
    }
}
// inverse of dif4 (up to the factor 4)
template <int MODE, class V>
__device__ __forceinline__ void dit4(V *x, int64_t N, int64_t M, const typename Cx<MODE>::Tw *tw,
                                     int tw_log2, int lgM2) {
    const int64_t h = M >> 1;
    for (int64_t t = threadIdx.x; t < N / 4; t += blockDim.x) {
        int64_t k = t & (h - 1);
        int64_t j = ((t - k) << 2) + k;
        V c0 = x[j], c1 = x[j + h], c2 = x[j + M], c3 = x[j + M + h];
        auto w1 = tw_get<MODE>(tw, tw_log2, k, lgM2);
        auto w2 = tw_get<MODE>(tw, tw_log2, k, lgM2 - 1);
        V t1 = twmul<true>(c1, w2);
        V b0 = cadd(c0, t1), b1 = csub(c0, t1);
        V t3 = twmul<true>(c3, w2);
        V b2 = cadd(c2, t3), b3 = csub(c2, t3);
        V t2 = twmul<true>(b2, w1);
        x[j] = cadd(b0, t2);
        x[j + M] = csub(b0, t2);
        V t4 = cmul_pi(twmul<true>(b3, w1));
        x[j + h] = cadd(b1, t4);
        x[j + M + h] = csub(b1, t4);
    }
}

// Forward DIF stages with half-sizes from Mhi down to Mlo (powers of two,
// Mhi >= Mlo >= 1) over N values, synchronising the block after each pass.
template <int MODE, class V>
__device__ void dif_range(V *x, int64_t N, int lgMhi, int lgMlo, const typename Cx<MODE>::Tw *tw,
                          int tw_log2) {
    int lg = lgMhi;
    if (((lgMhi - lgMlo + 1) & 1) != 0) {   // odd number of stages: one radix-2 first
        dif2<MODE>(x, N, (int64_t)1 << lg, tw, tw_log2, lg + 1);
        __syncthreads();
        lg--;
    }
    for (; lg > lgMlo; lg -= 2) {
        dif4<MODE>(x, N, (int64_t)1 << lg, tw, tw_log2, lg + 1);
        __syncthreads();
    }
}
// Inverse DIT stages with half-sizes from Mlo up to Mhi.
template <int MODE, class V>
__device__ void dit_range(V *x, int64_t N, int lgMlo, int lgMhi, const typename Cx<MODE>::Tw *tw,
                          int tw_log2) {
    int lg = lgMlo;
    // radix-4 pairs (lg, lg+1) first: the pair's stage order is h = 2^lg then 2^(lg+1)
    const int nst = lgMhi - lgMlo + 1;
    const int pairs = nst / 2;
    for (int p = 0; p < pairs; p++, lg += 2) {
        dit4<MODE>(x, N, (int64_t)1 << (lg + 1), tw, tw_log2, lg + 2);
        __syncthreads();
    }
    if (nst & 1) {
        dit2<MODE>(x, N, (int64_t)1 << lg, tw, tw_log2, lg + 1);
        __syncthreads();
    }
}

}  // namespace fft
}  // namespace aop
