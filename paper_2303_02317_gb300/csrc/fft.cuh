// fft.cuh -- FFT convolution engine for the linear advance of a row segment
// (the FFT-based linear-stencil step the trapezoid algorithm calls, Sec. 2.3
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
// Arithmetic modes:
//   MODE 0: FP64 complex values (double2), FP64 twiddles.
//   MODE 1: FP32 complex values (float2) carrying hi + i*lo of the FP64 input
//           (hi = fl32(x), lo = fl32(x - hi)); because the stencil power is
//           real, the real part of the result is conv(hi) and the imaginary
//           part conv(lo).  Twiddles and the kernel power are FP32 hi/lo pairs
//           applied with a compensated product.
//   MODE 2: double-float ("FP32 x 2") complex values: each component is an
//           unevaluated sum hi + lo of two FP32 numbers, added and multiplied
//           with error-free transformations (two-sum, two-product via FMA), so
//           the transform runs on the FP32 pipe with ~48-bit significands.
//
// Stage functions run on a thread group G (a warp or the whole block): G::rank()
// and G::size() give the thread's index and the group size, G::sync() the
// barrier between stages.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace aop {
namespace fft {

struct BlockGroup {
    __device__ static int rank() { return threadIdx.x; }
    __device__ static int size() { return blockDim.x; }
    __device__ static void sync() { __syncthreads(); }
};
struct WarpGroup {
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static int size() { return 32; }
    __device__ static void sync() { __syncwarp(); }
};

// double-float complex: x = re_hi, y = im_hi, z = re_lo, w = im_lo
struct df2 {
    float4 v;
};

template <int MODE> struct Cx;
template <> struct Cx<0> { using V = double2; using Tw = double2; using Sp = double2; };
template <> struct Cx<1> { using V = float2;  using Tw = float4;  using Sp = float4; };
template <> struct Cx<2> { using V = df2;     using Tw = float4;  using Sp = float4; };

// ------------------------------------------------------- double-float ops
// two-sum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// fast two-sum, |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}
// (ah + al) + (bh + bl) with the low parts summed before renormalising; the
// error is a few units of 2^-48 of |a| + |b|
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    fast_two_sum(s, e, rh, rl);
}
// (ah + al) * (bh + bl): exact high product through FMA, cross terms added
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float p = __fmul_rn(ah, bh);     // not fused into the sum below
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    fast_two_sum(p, e, rh, rl);
}

// w0 a + w1 (+ w2 c) for non-negative doubled-FP32 weights and values (the
// stencils of the lattices): high products exact through FMA, the low parts and
// the products' rounding errors summed once, one renormalisation (__fmul_rn keeps
// the compiler from fusing a product into the two-sum that follows).
__device__ __forceinline__ float2 df_dot2(float2 w0, float2 w1, float2 a, float2 b) {
    const float p0 = __fmul_rn(w0.x, a.x), p1 = __fmul_rn(w1.x, b.x);
    float e = fmaf(w0.x, a.x, -p0) + fmaf(w1.x, b.x, -p1);
    e = fmaf(w0.x, a.y, fmaf(w0.y, a.x, e));
    e = fmaf(w1.x, b.y, fmaf(w1.y, b.x, e));
    float s, t;
    two_sum(p0, p1, s, t);
    float h, l;
    fast_two_sum(s, t + e, h, l);
    return make_float2(h, l);
}
__device__ __forceinline__ float2 df_dot3(float2 w0, float2 w1, float2 w2, float2 a, float2 b, float2 c) {
    const float p0 = __fmul_rn(w0.x, a.x), p1 = __fmul_rn(w1.x, b.x), p2 = __fmul_rn(w2.x, c.x);
    float e = fmaf(w0.x, a.x, -p0) + fmaf(w1.x, b.x, -p1) + fmaf(w2.x, c.x, -p2);
    e = fmaf(w0.x, a.y, fmaf(w0.y, a.x, e));
    e = fmaf(w1.x, b.y, fmaf(w1.y, b.x, e));
    e = fmaf(w2.x, c.y, fmaf(w2.y, c.x, e));
    float s, t, s2, t2;
    two_sum(p0, p1, s, t);
    two_sum(s, p2, s2, t2);
    float h, l;
    fast_two_sum(s2, (t + t2) + e, h, l);
    return make_float2(h, l);
}
// a >= b for normalised doubled-FP32 values
__device__ __forceinline__ bool df_ge(float2 a, float2 b) { return a.x > b.x || (a.x == b.x && a.y >= b.y); }
// the nearest doubled-FP32 value of an FP64 number
__device__ __forceinline__ float2 df_from(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// ------------------------------------------------------------- complex ops
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// Transform sums keep the low part unnormalised (the exact two-sum error of
// the high parts plus the low parts): the next twiddle product renormalises,
// and the extraction adds hi + lo.
__device__ __forceinline__ void df_add_lazy(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float e;
    two_sum(ah, bh, rh, e);
    rl = e + (al + bl);
}
__device__ __forceinline__ df2 cadd(df2 a, df2 b) {
    df2 r;
    df_add_lazy(a.v.x, a.v.z, b.v.x, b.v.z, r.v.x, r.v.z);
    df_add_lazy(a.v.y, a.v.w, b.v.y, b.v.w, r.v.y, r.v.w);
    return r;
}
__device__ __forceinline__ df2 csub(df2 a, df2 b) {
    df2 r;
    df_add_lazy(a.v.x, a.v.z, -b.v.x, -b.v.z, r.v.x, r.v.z);
    df_add_lazy(a.v.y, a.v.w, -b.v.y, -b.v.w, r.v.y, r.v.w);
    return r;
}
// multiply by -i and by +i
__device__ __forceinline__ double2 cmul_mi(double2 a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ double2 cmul_pi(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 cmul_pi(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ df2 cmul_mi(df2 a) { df2 r; r.v = make_float4(a.v.y, -a.v.x, a.v.w, -a.v.z); return r; }
__device__ __forceinline__ df2 cmul_pi(df2 a) { df2 r; r.v = make_float4(-a.v.y, a.v.x, -a.v.w, a.v.z); return r; }

// complex conjugate and halving (exact)
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ df2 cconj(df2 a) { df2 r; r.v = make_float4(a.v.x, -a.v.y, a.v.z, -a.v.w); return r; }
__device__ __forceinline__ double2 chalf(double2 a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
__device__ __forceinline__ df2 chalf(df2 a) {
    df2 r;
    r.v = make_float4(0.5f * a.v.x, 0.5f * a.v.y, 0.5f * a.v.z, 0.5f * a.v.w);
    return r;
}

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
// double-float complex product with a double-float twiddle (hi.x, hi.y, lo.x, lo.y):
// each real part is p1 -+ p2 with the high products exact through FMA; the
// products' low parts are summed unnormalised and the result renormalised once
template <bool CONJ>
__device__ __forceinline__ df2 twmul(df2 v, float4 w) {
    const float ch = w.x, cl = w.z;
    const float sh = CONJ ? -w.y : w.y, sl = CONJ ? -w.w : w.w;
    const float xr = v.v.x, xrl = v.v.z, xi = v.v.y, xil = v.v.w;
    // re = xr c - xi s
    const float p1 = __fmul_rn(xr, ch), p2 = __fmul_rn(xi, sh);
    float e1 = fmaf(xr, ch, -p1), e2 = fmaf(xi, sh, -p2);
    e1 = fmaf(xr, cl, fmaf(xrl, ch, e1));
    e2 = fmaf(xi, sl, fmaf(xil, sh, e2));
    float s, t;
    two_sum(p1, -p2, s, t);
    df2 r;
    fast_two_sum(s, t + (e1 - e2), r.v.x, r.v.z);
    // im = xr s + xi c
    const float q1 = __fmul_rn(xr, sh), q2 = __fmul_rn(xi, ch);
    float f1 = fmaf(xr, sh, -q1), f2 = fmaf(xi, ch, -q2);
    f1 = fmaf(xr, sl, fmaf(xrl, sh, f1));
    f2 = fmaf(xi, cl, fmaf(xil, ch, f2));
    two_sum(q1, q2, s, t);
    fast_two_sum(s, t + (f1 + f2), r.v.y, r.v.w);
    return r;
}

// Twiddle e^{-2 pi i k / 2^lg} for 0 <= k < 2^(lg-1): entry 2^(lg-1) + k of the
// per-level table (levels 1 .. tw_log2).
template <int MODE>
__device__ __forceinline__ typename Cx<MODE>::Tw tw_get(const typename Cx<MODE>::Tw *tab, int tw_log2,
                                                       int64_t k, int lg) {
    return __ldg(&tab[((int64_t)1 << (lg - 1)) + k]);    // level lg of the table, lg <= tw_log2
}

__device__ __forceinline__ uint32_t brev_n(uint32_t p, int lgN) {
    return lgN == 0 ? 0u : (__brev(p) >> (32 - lgN));
}

// ------------------------------------------- asynchronous global->shared copy
// cp.async with a source size: bytes past src_bytes are zero-filled, so the
// zero padding of a transform costs no global read.  Every copy of a tile is
// in flight at once; cp_async_wait() waits for this thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src, int src_bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem_src), "r"(src_bytes)
                     : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(s), "l"(gmem_src), "n"(BYTES),
                     "r"(src_bytes)
                     : "memory");
    }
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// --------------------------------------------------- in-place stage kernels
// A tile holds rows x 2^lgQ columns (row t, column q at x[(t << lgQ) + q]).
// Each column is a sub-transform of a longer transform whose consecutive rows
// lie 2^s_lo elements apart, column q at offset q0 + q; a stage of half-size
// M = 2^lgM rows then takes its twiddles from level lgM + s_lo + 1 at index
// (tm << s_lo) + q0 + q, tm the row offset inside the half.  A plain tile is
// one column (lgQ = s_lo = q0 = 0).  The group G cooperates on the tile; every
// range function ends with a group barrier.  Indices are 32-bit (transforms
// of at most 2^30 points).  One butterfly per thread at a time: two in flight
// (loaded together) measured slower, the larger butterfly code missing in the
// instruction cache.
struct Cols {
    int lgQ, s_lo, q0;
};

// radix-2 DIF step (half-size 2^lgM rows) over nb = rows * Q / 2 butterflies
template <int MODE, class G, class V>
__device__ __forceinline__ void dif2c(V *x, int nb, int lgM, Cols c, const typename Cx<MODE>::Tw *tw) {
    using Tw = typename Cx<MODE>::Tw;
    const int qm = (1 << c.lgQ) - 1, mm = (1 << lgM) - 1;
    const Tw *tl = tw + (1 << (lgM + c.s_lo)) + c.q0;
    const int st = 1 << (lgM + c.lgQ);
    for (int s = G::rank(); s < nb; s += G::size()) {
        const int pr = s >> c.lgQ, q = s & qm, tm = pr & mm;
        V *p = x + ((((pr - tm) << 1) + tm) << c.lgQ) + q;
        const Tw w = __ldg(tl + (tm << c.s_lo) + q);
        const V u = p[0], v = p[st];
        p[0] = cadd(u, v);
        p[st] = twmul<false>(csub(u, v), w);
    }
}
// radix-2 DIT step (half-size 2^lgM rows)
template <int MODE, class G, class V>
__device__ __forceinline__ void dit2c(V *x, int nb, int lgM, Cols c, const typename Cx<MODE>::Tw *tw) {
    using Tw = typename Cx<MODE>::Tw;
    const int qm = (1 << c.lgQ) - 1, mm = (1 << lgM) - 1;
    const Tw *tl = tw + (1 << (lgM + c.s_lo)) + c.q0;
    const int st = 1 << (lgM + c.lgQ);
    for (int s = G::rank(); s < nb; s += G::size()) {
        const int pr = s >> c.lgQ, q = s & qm, tm = pr & mm;
        V *p = x + ((((pr - tm) << 1) + tm) << c.lgQ) + q;
        const Tw w = __ldg(tl + (tm << c.s_lo) + q);
        const V u = p[0], v = twmul<true>(p[st], w);
        p[0] = cadd(u, v);
        p[st] = csub(u, v);
    }
}

// one radix-4 butterfly: its four values (rows t, t + h, t + M, t + M + h)
// and its two twiddles (levels lgM + s_lo + 1 and lgM + s_lo)
template <int MODE, class V>
struct Bf4 {
    V *p;
    V a0, a1, a2, a3;
    typename Cx<MODE>::Tw w1, w2;
};
template <int MODE, class V>
__device__ __forceinline__ Bf4<MODE, V> bf4_load(V *x, int s, int lgM, Cols c, int hs,
                                                const typename Cx<MODE>::Tw *t1,
                                                const typename Cx<MODE>::Tw *t2) {
    Bf4<MODE, V> b;
    const int qm = (1 << c.lgQ) - 1, hm = (1 << (lgM - 1)) - 1;
    const int pr = s >> c.lgQ, q = s & qm, tm = pr & hm;
    b.p = x + ((((pr - tm) << 2) + tm) << c.lgQ) + q;
    const int k = (tm << c.s_lo) + q;
    b.w1 = __ldg(t1 + k);
    b.w2 = __ldg(t2 + k);
    b.a0 = b.p[0];
    b.a1 = b.p[hs];
    b.a2 = b.p[2 * hs];
    b.a3 = b.p[3 * hs];
    return b;
}
// two DIF stages (half-sizes M and M/2) as one radix-4 butterfly
template <int MODE, class V>
__device__ __forceinline__ void bf4_dif(const Bf4<MODE, V> &b, int hs) {
    const V b0 = cadd(b.a0, b.a2), b2 = twmul<false>(csub(b.a0, b.a2), b.w1);
    const V b1 = cadd(b.a1, b.a3), b3 = cmul_mi(twmul<false>(csub(b.a1, b.a3), b.w1));
    b.p[0] = cadd(b0, b1);
    b.p[hs] = twmul<false>(csub(b0, b1), b.w2);
    b.p[2 * hs] = cadd(b2, b3);
    b.p[3 * hs] = twmul<false>(csub(b2, b3), b.w2);
}
// its inverse (DIT, half-sizes M/2 then M; up to the factor 4)
template <int MODE, class V>
__device__ __forceinline__ void bf4_dit(const Bf4<MODE, V> &b, int hs) {
    const V t1 = twmul<true>(b.a1, b.w2);
    const V b0 = cadd(b.a0, t1), b1 = csub(b.a0, t1);
    const V t3 = twmul<true>(b.a3, b.w2);
    const V b2 = cadd(b.a2, t3), b3 = csub(b.a2, t3);
    const V t2 = twmul<true>(b2, b.w1);
    b.p[0] = cadd(b0, t2);
    b.p[2 * hs] = csub(b0, t2);
    const V t4 = cmul_pi(twmul<true>(b3, b.w1));
    b.p[hs] = cadd(b1, t4);
    b.p[3 * hs] = csub(b1, t4);
}
// radix-4 step over nb = rows * Q / 4 butterflies, M = 2^lgM >= 2 rows
template <int MODE, class G, bool DIF, class V>
__device__ __forceinline__ void step4c(V *x, int nb, int lgM, Cols c, const typename Cx<MODE>::Tw *tw) {
    using Tw = typename Cx<MODE>::Tw;
    const Tw *t1 = tw + (1 << (lgM + c.s_lo)) + c.q0;
    const Tw *t2 = tw + (1 << (lgM - 1 + c.s_lo)) + c.q0;
    const int hs = 1 << (lgM - 1 + c.lgQ);
    for (int s = G::rank(); s < nb; s += G::size()) {
        const Bf4<MODE, V> A = bf4_load<MODE>(x, s, lgM, c, hs, t1, t2);
        if (DIF) bf4_dif(A, hs);
        else bf4_dit(A, hs);
    }
}

// Forward DIF stages with half-sizes from 2^lgMhi down to 2^lgMlo rows on a
// tile of 2^lgR rows, a group barrier after each pass.  The range functions
// are kept out of line: every transform of a mode then runs one copy of the
// butterfly code, which with the walker's base cases must stay inside the
// SM's instruction cache (inlined at each call site, instruction fetch became
// the largest stall of the pricing kernel).
template <int MODE, class G, class V>
__device__ __noinline__ void dif_cols(V *x, int lgR, int lgMhi, int lgMlo, Cols c, const typename Cx<MODE>::Tw *tw) {
    int lg = lgMhi;
    if (((lgMhi - lgMlo + 1) & 1) != 0) {   // odd number of stages: one radix-2 first
        dif2c<MODE, G>(x, 1 << (lgR + c.lgQ - 1), lg, c, tw);
        G::sync();
        lg--;
    }
    for (; lg > lgMlo; lg -= 2) {
        step4c<MODE, G, true>(x, 1 << (lgR + c.lgQ - 2), lg, c, tw);
        G::sync();
    }
}
// Inverse DIT stages with half-sizes from 2^lgMlo up to 2^lgMhi rows.
template <int MODE, class G, class V>
__device__ __noinline__ void dit_cols(V *x, int lgR, int lgMlo, int lgMhi, Cols c, const typename Cx<MODE>::Tw *tw) {
    int lg = lgMlo;
    const int nst = lgMhi - lgMlo + 1;
    for (int p = 0; p < nst / 2; p++, lg += 2) {
        step4c<MODE, G, false>(x, 1 << (lgR + c.lgQ - 2), lg + 1, c, tw);
        G::sync();
    }
    if (nst & 1) {
        dit2c<MODE, G>(x, 1 << (lgR + c.lgQ - 1), lg, c, tw);
        G::sync();
    }
}
// The same stage ranges as radix-2 steps only: a transform schedule the
// autotuner may pick.  Separate out-of-line copies, so that the radix-4 code
// the default schedule runs is unchanged (the pricing kernel is sensitive to
// the size of its hot code).
template <int MODE, class G, class V>
__device__ __noinline__ void dif_cols_r2(V *x, int lgR, int lgMhi, int lgMlo, Cols c, const typename Cx<MODE>::Tw *tw) {
    for (int lg = lgMhi; lg >= lgMlo; lg--) {
        dif2c<MODE, G>(x, 1 << (lgR + c.lgQ - 1), lg, c, tw);
        G::sync();
    }
}
template <int MODE, class G, class V>
__device__ __noinline__ void dit_cols_r2(V *x, int lgR, int lgMlo, int lgMhi, Cols c, const typename Cx<MODE>::Tw *tw) {
    for (int lg = lgMlo; lg <= lgMhi; lg++) {
        dit2c<MODE, G>(x, 1 << (lgR + c.lgQ - 1), lg, c, tw);
        G::sync();
    }
}
// Whole transforms of a plain tile of 2^lgN points (r2: radix-2 steps only).
template <int MODE, class G, class V>
__device__ void dif_all(V *x, int lgN, const typename Cx<MODE>::Tw *tw, int r2 = 0) {
    if (r2) dif_cols_r2<MODE, G>(x, lgN, lgN - 1, 0, Cols{0, 0, 0}, tw);
    else dif_cols<MODE, G>(x, lgN, lgN - 1, 0, Cols{0, 0, 0}, tw);
}
template <int MODE, class G, class V>
__device__ void dit_all(V *x, int lgN, const typename Cx<MODE>::Tw *tw, int r2 = 0) {
    if (r2) dit_cols_r2<MODE, G>(x, lgN, 0, lgN - 1, Cols{0, 0, 0}, tw);
    else dit_cols<MODE, G>(x, lgN, 0, lgN - 1, Cols{0, 0, 0}, tw);
}

// ------------------------------------------------- value conversions by mode
template <int MODE> __device__ __forceinline__ typename Cx<MODE>::V load_split(double x);
template <> __device__ __forceinline__ double2 load_split<0>(double x) { return make_double2(x, 0.0); }
template <> __device__ __forceinline__ float2 load_split<1>(double x) {
    float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}
template <> __device__ __forceinline__ df2 load_split<2>(double x) {
    float hi = (float)x;
    df2 r;
    r.v = make_float4(hi, 0.f, (float)(x - (double)hi), 0.f);
    return r;
}
__device__ __forceinline__ double unsplit(double2 v, double invN) { return v.x * invN; }
__device__ __forceinline__ double unsplit(float2 v, double invN) { return ((double)v.x + (double)v.y) * invN; }
__device__ __forceinline__ double unsplit(df2 v, double invN) { return ((double)v.v.x + (double)v.v.z) * invN; }

// ----------------------------------------------------- stored row values
// Row values between transforms.  MODE 0 stores FP64.  MODES 1 and 2 store
// an unevaluated pair of FP32 numbers (value = hi + lo, ~48 significant bits):
// a transform then reads and writes FP32 only, so the convolution path issues
// no FP64 instruction (on GB300 an FP64 instruction occupies the sub-partition's
// FP64 unit for ~64 cycles and would stall the FP64 base cases beside it).
template <int MODE> struct CellT { using T = float2; };
template <> struct CellT<0> { using T = double; };

__device__ __forceinline__ double cell_value(double c) { return c; }
__device__ __forceinline__ double cell_value(float2 c) { return (double)c.x + (double)c.y; }
template <int MODE> __device__ __forceinline__ typename CellT<MODE>::T make_cell(double v);
template <> __device__ __forceinline__ double make_cell<0>(double v) { return v; }
template <> __device__ __forceinline__ float2 make_cell<1>(double v) {
    float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
template <> __device__ __forceinline__ float2 make_cell<2>(double v) { return make_cell<1>(v); }

// cell -> transform value (moves only)
__device__ __forceinline__ double2 cell_to_v(double c) { return make_double2(c, 0.0); }
__device__ __forceinline__ float2 cell_to_v1(float2 c) { return c; }
__device__ __forceinline__ df2 cell_to_v2(float2 c) { df2 r; r.v = make_float4(c.x, 0.f, c.y, 0.f); return r; }
// transform value -> cell, scaled by 1/N (a power of two: exact in FP32)
__device__ __forceinline__ double v_to_cell(double2 v, double invN, float) { return v.x * invN; }
__device__ __forceinline__ float2 v_to_cell(float2 v, double, float s) { return make_float2(v.x * s, v.y * s); }
__device__ __forceinline__ float2 v_to_cell(df2 v, double, float s) { return make_float2(v.v.x * s, v.v.z * s); }

template <class V> __device__ __forceinline__ V czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ df2 czero<df2>() { df2 r; r.v = make_float4(0.f, 0.f, 0.f, 0.f); return r; }

// Kernel power entry for a bin from the band-limited half spectrum sp[0..mc]
// (entries beyond the band are zero; the upper half is the conjugate mirror).
template <int MODE>
__device__ __forceinline__ typename Cx<MODE>::V spec_mul(typename Cx<MODE>::V z, const typename Cx<MODE>::Sp *sp,
                                                         int mc, uint32_t m, uint32_t N) {
    uint32_t mm = (m <= N / 2) ? m : N - m;
    if ((int)mm > mc) return czero<typename Cx<MODE>::V>();
    typename Cx<MODE>::Sp s = sp[mm];
    return (m <= N / 2) ? twmul<false>(z, s) : twmul<true>(z, s);
}

}  // namespace fft
}  // namespace aop
