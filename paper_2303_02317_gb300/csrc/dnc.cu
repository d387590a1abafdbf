// dnc.cu -- the trapezoidal divide-and-conquer pricer (hot-path rows a2-a7).
//
// One CTA prices one option at a time (persistent grid over a device queue of
// options).  Its threads walk the recursion with an explicit stack:
//
//   calls (binomial Sec. 3.3, trinomial appendix "Algorithm for American call
//   option pricing under TOPM"): a row's red cells are the columns [c0, b]
//   (b = divider, Cor. 2.7); cells right of b are green and evaluated in
//   closed form.  solve(i0, c0, b, h) advances rows i0 -> i0-h in two halves;
//   each half computes the cells whose dependency cone lies inside the red
//   window with one FFT linear advance ("computing all red cells on rt / dw")
//   and recurses on the strip of width D*h_half next to the divider
//   ("trapezoid pbvt / svcw").  Heights h <= B are solved by the naive loop.
//   The triangle is cut into a chain of trapezoids whose heights follow the
//   red count of their first row ("Partitioning the Triangle into
//   Trapezoids"); a leftover triangle is solved naively.
//
//   put (Sec. 5.3): green cells are left of the divider f, red cells right of
//   it.  region(n, lo, hi, f, h) advances the window [lo, hi] of row n to
//   [lo+h, hi-h] of row n+h in two halves; each half recurses on the
//   sub-trapezoid of base [f-2g, f+2g] around the divider ("trapezoid eglj"),
//   computes the red cells right of it with one FFT advance ("trapezoid fbnl")
//   and evaluates the green cells left of it in closed form.  The triangle is a
//   chain of trapezoids of halving height.
//
// Warp 0 runs the FP64 base cases and the value-versus-payoff tests; all
// warps run the FFT convolutions (fft.cuh).  The kernel power s(theta)^h of
// every (height, transform length) pair is evaluated once per option in FP64
// on the band where |s|^h exceeds 2^-60 of its peak and cached.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace aop {

namespace {

constexpr int kThreadsD = 128;
constexpr int kSpecSlots = 64;
constexpr int kLeftoverCall = 64;   // rows solved naively at the root

struct SpecEntry {
    int32_t g;       // height (steps)
    int32_t lgN;     // transform length
    int32_t mc;      // band: bins 0..mc stored
    int32_t pad;
    int64_t off;     // entry offset in the arena
};

struct DncArgs {
    const Params *params;
    int64_t n;
    int B;                 // base-case height (power of two)
    int lg_nsmem;          // log2 of the shared-memory FFT capacity
    int64_t W_max;         // widest row (doubles)
    char *ws;
    int64_t ws_stride;     // bytes per CTA
    int64_t off_r0, off_mid, off_scr, off_spec;   // byte offsets inside a CTA slot
    int64_t mid_off[kMaxDepth];                   // doubles, relative to off_mid
    int64_t spec_cap;      // arena entries
    const void *tw;
    int tw_log2;
    double *prices;
    int32_t *status;
    int32_t *bnd;
    const int64_t *bnd_off;
    int *queue;
    int *err;
    aop_stats *stats;
    int64_t *opt_ns;       // per-option device time (nullable)
};

// a row segment in memory: the value of column x lives at p[x - base]
struct Buf {
    double *p;
    int64_t base;
    __device__ double &at(int64_t x) const { return p[x - base]; }
};

struct Counters {
    long long convs, fft_points, fft_flops, conv_in, conv_out, base_cells, gbytes;
};

template <int MODE>
struct Dnc {
    using V = typename fft::Cx<MODE>::V;
    using Tw = typename fft::Cx<MODE>::Tw;
    using Sp = typename fft::Cx<MODE>::Sp;

    const DncArgs &a;
    const Params &P;
    const ExpTables &E;
    V *sm;                  // shared FFT buffer (N_smem values)
    char *slot;             // this CTA's global workspace
    SpecEntry *cache;       // shared
    int *ncache;            // shared
    int64_t *arena_used;    // shared
    int32_t *bnd;           // divider output of this option (nullable)
    Counters &cnt;

    __device__ Dnc(const DncArgs &a_, const Params &P_, const ExpTables &E_, V *sm_, char *slot_,
                   SpecEntry *cache_, int *ncache_, int64_t *au, int32_t *bnd_, Counters &c)
        : a(a_), P(P_), E(E_), sm(sm_), slot(slot_), cache(cache_), ncache(ncache_), arena_used(au),
          bnd(bnd_), cnt(c) {}

    __device__ double *mid(int d) const {
        return (double *)(slot + a.off_mid) + a.mid_off[d];
    }
    __device__ V *scratch() const { return (V *)(slot + a.off_scr); }
    __device__ Sp *arena() const { return (Sp *)(slot + a.off_spec); }
    __device__ const Tw *tw() const { return (const Tw *)a.tw; }

    __device__ void record(int64_t row, int32_t v) const {
        if (bnd) bnd[row] = v;
    }

    // ---------------------------------------------------------- kernel power
    __device__ int band_mc(int64_t g, int64_t N) const {
        const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        double kap = 4.0 * (w0 * w1 + (P.nw == 3 ? w1 * w2 : 0.0)) / (P.wsum * P.wsum);
        double need = 83.2 / ((double)g * kap);
        if (!(kap > 0) || need >= 1.0) return (int)(N / 2);
        double th2 = asin(sqrt(need));               // theta_c / 2
        double mc = (double)N * th2 / 3.141592653589793 + 2.0;
        return (int)min((double)(N / 2), ceil(mc));
    }

    // s(theta_m)^g for m in [0, mc]: computed in FP64 (magnitude through
    // log1p of the exactly formed 1 - |s/s(0)|^2, phase reduced in FP64).
    __device__ void compute_spectrum(Sp *dst, int64_t g, int lgN, int mc) const {
        const double N = (double)((int64_t)1 << lgN);
        const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        const double lws = log(P.wsum);
        const double inv2 = 1.0 / (P.wsum * P.wsum);
        const double gd = (double)g;
        for (int m = threadIdx.x; m <= mc; m += blockDim.x) {
            double sh, ch;
            sincospi((double)m / N, &sh, &ch);
            const double s1 = 2.0 * sh * ch, c1 = 1.0 - 2.0 * sh * sh;
            double re, im, dl;
            if (P.nw == 2) {
                re = w0 + w1 * c1;
                im = w1 * s1;
                dl = 4.0 * w0 * w1 * sh * sh * inv2;
            } else if (P.o_min == 0) {
                const double s2 = 2.0 * s1 * c1, c2 = 1.0 - 2.0 * s1 * s1;
                re = w0 + w1 * c1 + w2 * c2;
                im = w1 * s1 + w2 * s2;
                dl = 4.0 * ((w0 * w1 + w1 * w2) * sh * sh + w0 * w2 * s1 * s1) * inv2;
            } else {
                re = w1 + (w0 + w2) * c1;
                im = (w2 - w0) * s1;
                dl = 4.0 * ((w0 * w1 + w1 * w2) * sh * sh + w0 * w2 * s1 * s1) * inv2;
            }
            // 1 - |s/s(0)|^2 lies in [0, 1]; rounding can step outside when
            // |s(pi)| vanishes (e.g. p = 1/2), where the power is zero anyway
            dl = fmin(fmax(dl, 0.0), 1.0);
            double lm = (dl >= 1.0) ? -INFINITY : gd * (lws + 0.5 * log1p(-dl));
            double ph = gd * atan2(im, re);
            // reduce the phase to [-pi, pi] in units of pi
            double phpi = ph * 0.3183098861837907;
            phpi -= 2.0 * rint(0.5 * phpi);
            double sp, cp;
            sincospi(phpi, &sp, &cp);
            double mag = (lm < -745.0) ? 0.0 : exp(lm);
            double vr = mag * cp, vi = mag * sp;
            if constexpr (MODE == 0) {
                dst[m] = make_double2(vr, vi);
            } else {
                float hr = (float)vr, hi_ = (float)vi;
                dst[m] = make_float4(hr, hi_, (float)(vr - (double)hr), (float)(vi - (double)hi_));
            }
        }
    }

    // Find or build the cached spectrum; returns (pointer, mc) through refs.
    // Called by all threads (uniform); ends with a block barrier.
    __device__ const Sp *spectrum(int64_t g, int lgN, int &mc_out) {
        __shared__ int s_idx;
        __shared__ int s_build;
        if (threadIdx.x == 0) {
            int idx = -1;
            for (int i = 0; i < *ncache; i++)
                if (cache[i].g == (int32_t)g && cache[i].lgN == lgN) { idx = i; break; }
            s_build = 0;
            if (idx < 0) {
                int mc = band_mc(g, (int64_t)1 << lgN);
                if (*ncache >= kSpecSlots || *arena_used + mc + 1 > a.spec_cap) {
                    *ncache = 0;           // evict everything
                    *arena_used = 0;
                }
                idx = (*ncache)++;
                cache[idx].g = (int32_t)g;
                cache[idx].lgN = lgN;
                cache[idx].mc = mc;
                cache[idx].off = *arena_used;
                *arena_used += mc + 1;
                s_build = 1;
            }
            s_idx = idx;
        }
        __syncthreads();
        const SpecEntry e = cache[s_idx];
        Sp *p = arena() + e.off;
        if (s_build) {
            compute_spectrum(p, g, lgN, e.mc);
            __threadfence_block();
        }
        __syncthreads();
        mc_out = e.mc;
        return p;
    }

    // ---------------------------------------------------------- conv helpers
    __device__ static V load_split(double x) {
        if constexpr (MODE == 0) {
            return make_double2(x, 0.0);
        } else {
            float hi = (float)x;
            return make_float2(hi, (float)(x - (double)hi));
        }
    }
    __device__ static double unsplit(V v, double invN) {
        if constexpr (MODE == 0) return v.x * invN;
        else return ((double)v.x + (double)v.y) * invN;
    }
    __device__ static V spec_mul(V z, const Sp *sp, int mc, uint32_t m, uint32_t N) {
        uint32_t mm = (m <= N / 2) ? m : N - m;
        if ((int)mm > mc) {
            V zero;
            zero.x = 0; zero.y = 0;
            return zero;
        }
        Sp s = sp[mm];
        return (m <= N / 2) ? fft::twmul<false>(z, s) : fft::twmul<true>(z, s);
    }

    // Linear advance: out[y] = sum_t c_t in[y + o_min g + t] for y in
    // [x_lo - o_min g, x_hi - (o_min + nw - 1) g] (the window fully inside the
    // input [x_lo, x_hi]).  All threads call it; ends with a barrier.
    __device__ void conv(const Buf in, int64_t x_lo, int64_t x_hi, const Buf out, int64_t g) {
        const int64_t W = x_hi - x_lo + 1;
        const int64_t span = (int64_t)(P.nw - 1) * g;
        const int64_t y_lo = x_lo - (int64_t)P.o_min * g;
        const int64_t nout = W - span;
        if (nout <= 0) return;
        int lgN = ilog2_ceil(W);
        if (lgN < 2) lgN = 2;
        const int64_t N = (int64_t)1 << lgN;
        int mc;
        const Sp *sp = spectrum(g, lgN, mc);
        const double invN = 1.0 / (double)N;
        if (threadIdx.x == 0) {
            cnt.convs++;
            cnt.fft_points += 2 * N;
            cnt.fft_flops += 2 * 5 * N * lgN;
            cnt.conv_in += W;
            cnt.conv_out += nout;
        }
        if (lgN <= a.lg_nsmem) {
            for (int64_t e = threadIdx.x; e < N; e += blockDim.x)
                sm[e] = load_split(e < W ? in.at(x_lo + e) : 0.0);
            __syncthreads();
            fft::dif_range<MODE>(sm, N, lgN - 1, 0, tw(), a.tw_log2);
            for (int64_t p = threadIdx.x; p < N; p += blockDim.x)
                sm[p] = spec_mul(sm[p], sp, mc, fft::brev_n((uint32_t)p, lgN), (uint32_t)N);
            __syncthreads();
            fft::dit_range<MODE>(sm, N, 0, lgN - 1, tw(), a.tw_log2);
            const int64_t off = y_lo - x_lo;   // output y sits at transform index y - x_lo
            for (int64_t t = threadIdx.x; t < nout; t += blockDim.x)
                out.at(y_lo + t) = unsplit(sm[off + t], invN);
            __syncthreads();
        } else {
            conv_global(in, x_lo, W, out, y_lo, nout, lgN, sp, mc, invN);
        }
    }

    // Three passes through global scratch for N > shared capacity:
    //   A: the outer DIF stages (half-sizes N/2 .. N2) on the strided groups
    //      {q + t N2}, loading (and splitting) the FP64 input;
    //   B: per contiguous block of N2: inner DIF stages, kernel-power product,
    //      inner DIT stages;
    //   C: the outer DIT stages on the strided groups, then the extraction.
    __device__ void conv_global(const Buf in, int64_t x_lo, int64_t W, const Buf out, int64_t y_lo,
                                int64_t nout, int lgN, const Sp *sp, int mc, double invN) {
        const int lg2 = a.lg_nsmem;          // block length N2
        const int lg1 = lgN - lg2;           // number of blocks N1
        const int64_t N = (int64_t)1 << lgN, N1 = (int64_t)1 << lg1, N2 = (int64_t)1 << lg2;
        const int64_t Q = N2 >> lg1;         // columns per tile (>= 1)
        V *scr = scratch();
        const Tw *T = tw();
        const int twl = a.tw_log2;
        if (threadIdx.x == 0) cnt.gbytes += (int64_t)sizeof(V) * N * 4 + 8 * (W + nout);
        // ---- pass A
        for (int64_t q0 = 0; q0 < N2; q0 += Q) {
            for (int64_t s = threadIdx.x; s < N1 * Q; s += blockDim.x) {
                int64_t t = s / Q, q = s - t * Q;
                int64_t e = q0 + q + t * N2;
                sm[s] = load_split(e < W ? in.at(x_lo + e) : 0.0);
            }
            __syncthreads();
            for (int lgm = lg1 - 1; lgm >= 0; lgm--) {      // t-space half size m
                const int64_t m = (int64_t)1 << lgm;
                const int lgM2 = lgm + lg2 + 1;               // 2M = 2 m N2
                for (int64_t s = threadIdx.x; s < (N1 / 2) * Q; s += blockDim.x) {
                    int64_t pr = s / Q, q = s - pr * Q;
                    int64_t tm = pr & (m - 1);
                    int64_t t = ((pr - tm) << 1) + tm;
                    int64_t kk = q0 + q + tm * N2;            // e mod 2M
                    V u = sm[t * Q + q], v = sm[(t + m) * Q + q];
                    sm[t * Q + q] = fft::cadd(u, v);
                    sm[(t + m) * Q + q] = fft::twmul<false>(fft::csub(u, v),
                                                            fft::tw_get<MODE>(T, twl, kk, lgM2));
                }
                __syncthreads();
            }
            for (int64_t s = threadIdx.x; s < N1 * Q; s += blockDim.x) {
                int64_t t = s / Q, q = s - t * Q;
                scr[q0 + q + t * N2] = sm[s];
            }
            __syncthreads();
        }
        // ---- pass B
        for (int64_t b = 0; b < N1; b++) {
            V *blk = scr + b * N2;
            for (int64_t s = threadIdx.x; s < N2; s += blockDim.x) sm[s] = blk[s];
            __syncthreads();
            fft::dif_range<MODE>(sm, N2, lg2 - 1, 0, T, twl);
            for (int64_t s = threadIdx.x; s < N2; s += blockDim.x)
                sm[s] = spec_mul(sm[s], sp, mc, fft::brev_n((uint32_t)(b * N2 + s), lgN), (uint32_t)N);
            __syncthreads();
            fft::dit_range<MODE>(sm, N2, 0, lg2 - 1, T, twl);
            for (int64_t s = threadIdx.x; s < N2; s += blockDim.x) blk[s] = sm[s];
            __syncthreads();
        }
        // ---- pass C
        const int64_t off = y_lo - x_lo;
        for (int64_t q0 = 0; q0 < N2; q0 += Q) {
            for (int64_t s = threadIdx.x; s < N1 * Q; s += blockDim.x) {
                int64_t t = s / Q, q = s - t * Q;
                sm[s] = scr[q0 + q + t * N2];
            }
            __syncthreads();
            for (int lgm = 0; lgm < lg1; lgm++) {
                const int64_t m = (int64_t)1 << lgm;
                const int lgM2 = lgm + lg2 + 1;
                for (int64_t s = threadIdx.x; s < (N1 / 2) * Q; s += blockDim.x) {
                    int64_t pr = s / Q, q = s - pr * Q;
                    int64_t tm = pr & (m - 1);
                    int64_t t = ((pr - tm) << 1) + tm;
                    int64_t kk = q0 + q + tm * N2;
                    V u = sm[t * Q + q];
                    V v = fft::twmul<true>(sm[(t + m) * Q + q], fft::tw_get<MODE>(T, twl, kk, lgM2));
                    sm[t * Q + q] = fft::cadd(u, v);
                    sm[(t + m) * Q + q] = fft::csub(u, v);
                }
                __syncthreads();
            }
            for (int64_t s = threadIdx.x; s < N1 * Q; s += blockDim.x) {
                int64_t t = s / Q, q = s - t * Q;
                int64_t e = q0 + q + t * N2;
                int64_t k = e - off;
                if (k >= 0 && k < nout) out.at(y_lo + k) = unsplit(sm[s], invN);
            }
            __syncthreads();
        }
    }

    // ------------------------------------------------------ naive base cases
    // Call: rows i0-1 .. i0-h from the red cells [c0, b] of row i0 (in), red
    // cells of row i0-h written to out; returns the new divider.  Warp 0 only;
    // the caller brackets it with barriers.  Values live in shared memory.
    __device__ int64_t naive_call(int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf in,
                                  const Buf out) {
        const int lane = threadIdx.x & 31;
        double *cur = (double *)sm;
        const int64_t cap = ((int64_t)sizeof(V) << a.lg_nsmem) / (2 * sizeof(double));
        double *nxt = cur + cap;
        const int D = P.D;
        const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        if (b - c0 + 1 + D > cap) {          // never expected: window wider than the buffer
            if (lane == 0) set_error(a.err, AOP_EINTERNAL);
            return b;
        }
        for (int64_t x = c0 + lane; x <= b; x += 32) cur[x - c0] = in.at(x);
        __syncwarp();
        long long cells = 0;
        for (int64_t k = 1; k <= h; k++) {
            const int64_t i = i0 - k;
            const int64_t bp = b;
            if (bp < c0) {
                if (lane == 0) record(i, (int32_t)(c0 - 1));
                continue;
            }
            const int64_t top = min(bp, (int64_t)D * i);
            for (int64_t x = c0 + lane; x <= top; x += 32) {
                double v0 = cur[x - c0];
                double v1 = (x + 1 <= bp) ? cur[x + 1 - c0] : exercise(P, E, ex_index(P, i + 1, x + 1));
                double c = w0 * v0 + w1 * v1;
                if (D == 2) {
                    double v2 = (x + 2 <= bp) ? cur[x + 2 - c0] : exercise(P, E, ex_index(P, i + 1, x + 2));
                    c += w2 * v2;
                }
                nxt[x - c0] = c;
                cells++;
            }
            __syncwarp();
            int64_t bn;
            if (bp - 1 >= (int64_t)D * i) {
                bn = (int64_t)D * i;
            } else {
                // value-versus-payoff test at the previous divider (Cor. 2.7)
                const double cont = nxt[bp - c0];
                bn = (cont >= exercise(P, E, ex_index(P, i, bp))) ? bp : bp - 1;
            }
            b = bn;
            if (lane == 0) record(i, (int32_t)(b >= c0 ? b : c0 - 1));
            double *t = cur; cur = nxt; nxt = t;
            __syncwarp();
        }
        for (int64_t x = c0 + lane; x <= b; x += 32) out.at(x) = cur[x - c0];
        cells = __reduce_add_sync(0xffffffffu, (unsigned)cells);
        if (lane == 0) cnt.base_cells += cells;
        return b;
    }

    // Put: rows n+1 .. n+h over the window [lo, hi] of row n with divider f;
    // red cells (> f) come from in; writes the red cells of row n+h to out.
    __device__ int64_t naive_put(int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h,
                                 const Buf in, const Buf out) {
        const int lane = threadIdx.x & 31;
        double *cur = (double *)sm;
        const int64_t cap = ((int64_t)sizeof(V) << a.lg_nsmem) / (2 * sizeof(double));
        double *nxt = cur + cap;
        const double wb = P.w[0], wc = P.w[1], wa = P.w[2];
        if (hi - lo + 1 > cap) {
            if (lane == 0) set_error(a.err, AOP_EINTERNAL);
            return f;
        }
        // full window values (green in closed form)
        for (int64_t x = lo + lane; x <= hi; x += 32)
            cur[x - lo] = (x <= f) ? exercise(P, E, ex_index(P, n, x)) : in.at(x);
        __syncwarp();
        long long cells = 0;
        int64_t L = lo, R = hi;
        for (int64_t k = 1; k <= h; k++) {
            const int64_t nl = L + 1, nr = R - 1;
            const int64_t fp = f;
            for (int64_t x = nl + lane; x <= nr; x += 32) {
                double c = wb * cur[x - 1 - lo] + wc * cur[x - lo] + wa * cur[x + 1 - lo];
                nxt[x - lo] = c;
                cells++;
            }
            __syncwarp();
            int64_t fn;
            if (fp >= nr + 1) fn = nr;
            else if (fp < nl) fn = fp;
            else {
                const double ex = exercise(P, E, ex_index(P, n + k, fp));
                fn = (ex > nxt[fp - lo]) ? fp : fp - 1;
            }
            f = fn;
            // green cells of the new row hold the payoff
            for (int64_t x = nl + lane; x <= min(f, nr); x += 32)
                nxt[x - lo] = exercise(P, E, ex_index(P, n + k, x));
            if (lane == 0) record(n + k, (f >= nl) ? (int32_t)f : (int32_t)AOP_BOUNDARY_NONE_PUT);
            double *t = cur; cur = nxt; nxt = t;
            L = nl; R = nr;
            __syncwarp();
        }
        for (int64_t x = max(L, f + 1) + lane; x <= R; x += 32) out.at(x) = cur[x - lo];
        cells = __reduce_add_sync(0xffffffffu, (unsigned)cells);
        if (lane == 0) cnt.base_cells += cells;
        return f;
    }

    // run naive_* on warp 0 and broadcast the divider
    __device__ int64_t base_call(int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf in, const Buf out) {
        __shared__ int64_t s_ret;
        __syncthreads();
        if (threadIdx.x < 32) {
            int64_t r = naive_call(i0, c0, b, h, in, out);
            if (threadIdx.x == 0) s_ret = r;
        }
        __syncthreads();
        return s_ret;
    }
    __device__ int64_t base_put(int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h, const Buf in,
                                const Buf out) {
        __shared__ int64_t s_ret;
        __syncthreads();
        if (threadIdx.x < 32) {
            int64_t r = naive_put(n, lo, hi, f, h, in, out);
            if (threadIdx.x == 0) s_ret = r;
        }
        __syncthreads();
        return s_ret;
    }

    __device__ void record_range(int64_t r0, int64_t r1, int32_t v) {
        if (!bnd) return;
        for (int64_t r = r0 + threadIdx.x; r <= r1; r += blockDim.x) bnd[r] = v;
    }

    // ------------------------------------------------------------ the call
    struct FrameC {
        int64_t i0, c0, b, h;
        Buf in, out;
        int depth, phase;
    };

    __device__ int64_t solve_call(int64_t i0, int64_t b, int64_t h, const Buf row) {
        FrameC st[kMaxDepth];
        int sp = 0;
        int64_t ret = 0;
        const int D = P.D;
        st[sp++] = FrameC{i0, 0, b, h, row, row, 0, 0};
        while (sp > 0) {
            FrameC &F = st[sp - 1];
            if (F.phase == 0) {
                if (F.b < F.c0) {
                    record_range(F.i0 - F.h, F.i0 - 1, (int32_t)(F.c0 - 1));
                    ret = F.c0 - 1;
                    sp--;
                    continue;
                }
                if (F.h <= a.B || F.depth + 1 >= kMaxDepth) {
                    ret = base_call(F.i0, F.c0, F.b, F.h, F.in, F.out);
                    sp--;
                    continue;
                }
                const int64_t h1 = F.h >> 1;
                const Buf M{mid(F.depth), F.c0};
                if (F.b - D * h1 >= F.c0) conv(F.in, F.c0, F.b, M, h1);
                const int64_t c1 = max(F.c0, F.b - D * h1 + 1);
                F.phase = 1;
                st[sp++] = FrameC{F.i0, c1, F.b, h1, F.in, M, F.depth + 1, 0};
            } else if (F.phase == 1) {
                const int64_t b1 = ret;
                const int64_t h1 = F.h >> 1, h2 = F.h - h1;
                const Buf M{mid(F.depth), F.c0};
                if (b1 - D * h2 >= F.c0) conv(M, F.c0, b1, F.out, h2);
                const int64_t c2 = max(F.c0, b1 - D * h2 + 1);
                F.phase = 2;
                st[sp++] = FrameC{F.i0 - h1, c2, b1, h2, M, F.out, F.depth + 1, 0};
            } else {
                sp--;
            }
        }
        return ret;
    }

    __device__ double price_call() {
        const int64_t T = P.T;
        const int D = P.D;
        const Buf row{(double *)(slot + a.off_r0), 0};
        __shared__ int s_b;
        // row T: red iff its payoff is <= 0 (continuation 0); row T-1 naive.
        if (threadIdx.x == 0) s_b = -1;
        __syncthreads();
        int bt = -1;
        for (int64_t j = threadIdx.x; j <= (int64_t)D * T; j += blockDim.x)
            if (0.0 >= exercise(P, E, ex_index(P, T, j))) bt = max(bt, (int)j);
        bt = __reduce_max_sync(0xffffffffu, bt);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_b, bt);
        __syncthreads();
        if (threadIdx.x == 0) record(T, s_b);
        __syncthreads();
        int64_t i = T - 1;
        if (threadIdx.x == 0) s_b = -1;
        __syncthreads();
        int br = -1;
        const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        for (int64_t j = threadIdx.x; j <= (int64_t)D * i; j += blockDim.x) {
            double c = w0 * fmax(exercise(P, E, ex_index(P, T, j)), 0.0) +
                       w1 * fmax(exercise(P, E, ex_index(P, T, j + 1)), 0.0);
            if (D == 2) c += w2 * fmax(exercise(P, E, ex_index(P, T, j + 2)), 0.0);
            row.at(j) = c;
            if (c >= exercise(P, E, ex_index(P, i, j))) br = max(br, (int)j);
        }
        br = __reduce_max_sync(0xffffffffu, br);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_b, br);
        __syncthreads();
        int64_t b = s_b;
        if (threadIdx.x == 0) record(i, (int32_t)b);
        __syncthreads();
        while (i > 0) {
            if (b < 0) {
                record_range(0, i - 1, -1);
                __syncthreads();
                return exercise(P, E, ex_index(P, 0, 0));
            }
            const int64_t avail = i - kLeftoverCall;
            if (avail < a.B) {
                b = base_call(i, 0, b, i, row, row);
                i = 0;
                break;
            }
            const int64_t w = b + 1;
            const int64_t want = max((int64_t)a.B, (w + D - 1) / D);
            int64_t h = a.B;
            while (2 * h <= want && 2 * h <= avail) h *= 2;
            b = solve_call(i, b, h, row);
            i -= h;
        }
        __syncthreads();
        if (b < 0) return exercise(P, E, ex_index(P, 0, 0));
        return row.at(0);
    }

    // ------------------------------------------------------------- the put
    struct FrameP {
        int64_t n, lo, hi, f, h;
        Buf in, out;
        int depth, phase;
    };

    __device__ int64_t solve_put(int64_t n0, int64_t lo0, int64_t hi0, int64_t f0, int64_t h0,
                                 const Buf row) {
        FrameP st[kMaxDepth];
        int sp = 0;
        int64_t ret = 0;
        st[sp++] = FrameP{n0, lo0, hi0, f0, h0, row, row, 0, 0};
        while (sp > 0) {
            FrameP &F = st[sp - 1];
            const int64_t h1 = F.h >> 1, h2 = F.h - h1;
            if (F.phase == 0) {
                if (F.f < F.lo) {        // no green cell in the window: one advance
                    conv(F.in, F.lo, F.hi, F.out, F.h);
                    record_range(F.n + 1, F.n + F.h, AOP_BOUNDARY_NONE_PUT);
                    ret = F.lo + F.h - 1;
                    sp--;
                    continue;
                }
                if (F.h <= a.B || F.depth + 1 >= kMaxDepth) {
                    ret = base_put(F.n, F.lo, F.hi, F.f, F.h, F.in, F.out);
                    sp--;
                    continue;
                }
                const Buf M{mid(F.depth), F.lo + h1};
                if (F.f + 1 + h1 <= F.hi - h1) conv(F.in, F.f + 1, F.hi, M, h1);
                const int64_t lo2 = max(F.lo, F.f - 2 * h1), hi2 = min(F.hi, F.f + 2 * h1);
                F.phase = 1;
                st[sp++] = FrameP{F.n, lo2, hi2, F.f, h1, F.in, M, F.depth + 1, 0};
            } else if (F.phase == 1) {
                const int64_t f1 = ret;
                const int64_t lo1 = F.lo + h1, hi1 = F.hi - h1;
                const Buf M{mid(F.depth), lo1};
                if (f1 < lo1) {
                    conv(M, lo1, hi1, F.out, h2);
                    record_range(F.n + h1 + 1, F.n + F.h, AOP_BOUNDARY_NONE_PUT);
                    ret = F.lo + F.h - 1;
                    sp--;
                    continue;
                }
                if (f1 + 1 + h2 <= hi1 - h2) conv(M, f1 + 1, hi1, F.out, h2);
                const int64_t lo2 = max(lo1, f1 - 2 * h2), hi2 = min(hi1, f1 + 2 * h2);
                F.phase = 2;
                st[sp++] = FrameP{F.n + h1, lo2, hi2, f1, h2, M, F.out, F.depth + 1, 0};
            } else {
                sp--;
            }
        }
        return ret;
    }

    __device__ double price_put() {
        const int64_t T = P.T;
        const Buf row{(double *)(slot + a.off_r0), -T};
        __shared__ int s_f;
        if (threadIdx.x == 0) s_f = INT32_MIN;
        __syncthreads();
        int fb = INT32_MIN;
        for (int64_t k = -T + threadIdx.x; k <= T; k += blockDim.x) {
            double e = exercise(P, E, ex_index(P, 0, k));
            row.at(k) = e > 0.0 ? e : 0.0;
            if (e > 0.0) fb = max(fb, (int)k);
        }
        fb = __reduce_max_sync(0xffffffffu, fb);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_f, fb);
        __syncthreads();
        if (threadIdx.x == 0) record(0, s_f);
        __syncthreads();
        // Row 1 over the whole row.  The divider theorem (k_n - k_{n+1} <= 1)
        // rests on the divider cell being green by the max at row n; at the
        // expiry row it is green by its payoff alone, so row 0 -> 1 may move
        // the divider arbitrarily far (e.g. r = 0: no cell stays green).
        if (threadIdx.x == 0) s_f = INT32_MIN;
        const Buf tmp{mid(0), -T};
        __syncthreads();
        fb = INT32_MIN;
        {
            const double wb = P.w[0], wc = P.w[1], wa = P.w[2];
            for (int64_t k = -(T - 1) + threadIdx.x; k <= T - 1; k += blockDim.x) {
                const double c = wb * row.at(k - 1) + wc * row.at(k) + wa * row.at(k + 1);
                const double e = exercise(P, E, ex_index(P, 1, k));
                const bool green = e > c;
                tmp.at(k) = green ? e : c;
                if (green) fb = max(fb, (int)k);
            }
        }
        fb = __reduce_max_sync(0xffffffffu, fb);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_f, fb);
        __syncthreads();
        for (int64_t k = -(T - 1) + threadIdx.x; k <= T - 1; k += blockDim.x) row.at(k) = tmp.at(k);
        if (threadIdx.x == 0) record(1, s_f);
        int64_t f = (s_f == INT32_MIN) ? -T - 1 : s_f;
        __syncthreads();
        int64_t n = 1;
        while (T - n > 0) {
            const int64_t R = T - n;
            if (f >= R) {                // every remaining cell is green
                for (int64_t r = n + 1 + threadIdx.x; r <= T; r += blockDim.x)
                    if (bnd) bnd[r] = (int32_t)(T - r);
                __syncthreads();
                return P.out_scale * exercise(P, E, ex_index(P, T, 0));
            }
            if (R / 2 < a.B || R <= 2 * a.B) {
                f = base_put(n, -R, R, f, R, row, row);
                n = T;
                break;
            }
            int64_t h = a.B;
            while (2 * h <= R / 2) h *= 2;
            f = solve_put(n, -R, R, f, h, row);
            n += h;
        }
        __syncthreads();
        if (f >= 0) return P.out_scale * exercise(P, E, ex_index(P, T, 0));
        return P.out_scale * row.at(0);
    }
};

template <int MODE>
__global__ void __launch_bounds__(kThreadsD) dnc_kernel(const __grid_constant__ DncArgs a)
{
    using V = typename fft::Cx<MODE>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ExpTables E;
    __shared__ Params sP;
    __shared__ SpecEntry cache[kSpecSlots];
    __shared__ int ncache;
    __shared__ int64_t arena_used;
    __shared__ int s_opt;
    V *sm = (V *)smem_raw;
    char *slot = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    Counters cnt{0, 0, 0, 0, 0, 0, 0};
    for (;;) {
        if (threadIdx.x == 0) s_opt = atomicAdd(a.queue, 1);
        __syncthreads();
        const int64_t o = s_opt;
        if (o >= a.n) break;
        if (threadIdx.x == 0) {
            sP = a.params[o];
            ncache = 0;
            arena_used = 0;
        }
        __syncthreads();
        if (sP.status != AOP_OK) {
            if (threadIdx.x == 0) a.prices[o] = __longlong_as_double(0x7ff8000000000000ll);
            __syncthreads();
            continue;
        }
        build_exp_tables(sP, E);
        __syncthreads();
        uint64_t t_start = 0;
        if (threadIdx.x == 0 && a.opt_ns) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
        int32_t *bnd = a.bnd ? a.bnd + a.bnd_off[o] : nullptr;
        Dnc<MODE> d(a, sP, E, sm, slot, cache, &ncache, &arena_used, bnd, cnt);
        double price = (sP.model == AOP_BSM_PUT) ? d.price_put() : d.price_call();
        if (threadIdx.x == 0) {
            a.prices[o] = price;
            if (a.opt_ns) {
                uint64_t t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                a.opt_ns[o] = (int64_t)(t_end - t_start);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && a.stats) {
        atomicAdd((unsigned long long *)&a.stats->convolutions, (unsigned long long)cnt.convs);
        atomicAdd((unsigned long long *)&a.stats->fft_points, (unsigned long long)cnt.fft_points);
        atomicAdd((unsigned long long *)&a.stats->fft_flops, (unsigned long long)cnt.fft_flops);
        atomicAdd((unsigned long long *)&a.stats->conv_inputs, (unsigned long long)cnt.conv_in);
        atomicAdd((unsigned long long *)&a.stats->conv_outputs, (unsigned long long)cnt.conv_out);
        atomicAdd((unsigned long long *)&a.stats->global_fft_bytes, (unsigned long long)cnt.gbytes);
    }
    if ((threadIdx.x & 31) == 0 && threadIdx.x == 0 && a.stats)
        atomicAdd((unsigned long long *)&a.stats->basecase_cells, (unsigned long long)cnt.base_cells);
}

// ------------------------------------------------------------ layout/launch
struct Layout {
    int64_t W_max, N_max, spec_cap;
    int64_t off_r0, off_mid, off_scr, off_spec, stride;
    int64_t mid_off[kMaxDepth];
    int lg_nsmem, tw_log2;
};

Layout make_layout(int method, int64_t T_max, int B) {
    Layout L;
    L.W_max = 2 * T_max + 1;
    L.N_max = (int64_t)1 << ilog2_ceil(L.W_max);
    L.lg_nsmem = (method == AOP_FFT_FP64) ? 11 : 12;   // 32 KiB of shared memory
    L.tw_log2 = max(ilog2_ceil(L.N_max), L.lg_nsmem + 1);
    const int64_t vsz = (method == AOP_FFT_FP64) ? 16 : 8;
    const int64_t ssz = 16;
    // one spectrum holds at most N/2 + 1 bins: the arena always fits the largest
    L.spec_cap = std::max<int64_t>(1 << 17, L.N_max / 2 + 2);
    int64_t off = 0;
    L.off_r0 = off;
    off += ((L.W_max + 64) * 8 + 255) & ~255ll;
    L.off_mid = off;
    int64_t m = 0;
    for (int d = 0; d < kMaxDepth; d++) {
        L.mid_off[d] = m;
        int64_t cap = (d == 0) ? L.W_max + 8 : (L.W_max >> d) + 4ll * B + 16;
        m += (cap + 31) & ~31ll;
    }
    off += (m * 8 + 255) & ~255ll;
    L.off_scr = off;
    off += (L.N_max * vsz + 255) & ~255ll;
    L.off_spec = off;
    off += (L.spec_cap * ssz + 255) & ~255ll;
    L.stride = off;
    return L;
}

int g_sms_cache[64];

int sm_count(int device) {
    if (device < 0 || device >= 64) device = 0;
    if (g_sms_cache[device] == 0) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        g_sms_cache[device] = sms > 0 ? sms : 1;
    }
    return g_sms_cache[device];
}

}  // namespace

size_t dnc_workspace_bytes(int method, int64_t n, int64_t T_max, int base_case, int *grid_out, int device)
{
    Layout L = make_layout(method, T_max, base_case);
    int64_t grid = std::min<int64_t>(n, (int64_t)sm_count(device) * 4);
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    return (size_t)(grid * L.stride + 4096);
}

cudaError_t run_dnc(int method, int64_t n, const Params *d_params, int64_t T_max, int base_case,
                    void *ws, size_t ws_bytes, const void *d_tw, int tw_log2, double *d_prices,
                    int32_t *d_status, int32_t *d_bnd, const int64_t *d_bnd_off,
                    aop_stats *d_stats, int *d_err, int64_t *d_opt_ns, int device, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    Layout L = make_layout(method, T_max, base_case);
    if (tw_log2 < L.tw_log2) return cudaErrorInvalidValue;
    int64_t grid = std::min<int64_t>(n, (int64_t)sm_count(device) * 4);
    // the queue counter lives at the end of the workspace
    const size_t need = (size_t)(grid * L.stride) + 4096;
    if (ws_bytes < need) {
        grid = (int64_t)((ws_bytes - 4096) / L.stride);
        if (grid < 1) return cudaErrorMemoryAllocation;
    }
    char *base = (char *)ws;
    int *queue = (int *)(base + grid * L.stride);
    cudaMemsetAsync(queue, 0, sizeof(int), s);
    DncArgs a;
    a.params = d_params;
    a.n = n;
    a.B = base_case;
    a.lg_nsmem = L.lg_nsmem;
    a.W_max = L.W_max;
    a.ws = base;
    a.ws_stride = L.stride;
    a.off_r0 = L.off_r0;
    a.off_mid = L.off_mid;
    a.off_scr = L.off_scr;
    a.off_spec = L.off_spec;
    for (int d = 0; d < kMaxDepth; d++) a.mid_off[d] = L.mid_off[d];
    a.spec_cap = L.spec_cap;
    a.tw = d_tw;
    a.tw_log2 = tw_log2;
    a.prices = d_prices;
    a.status = d_status;
    a.bnd = d_bnd;
    a.bnd_off = d_bnd_off;
    a.queue = queue;
    a.err = d_err;
    a.stats = d_stats;
    a.opt_ns = d_opt_ns;
    const size_t smem = (size_t)((method == AOP_FFT_FP64) ? 16 : 8) << L.lg_nsmem;
    if (method == AOP_FFT_FP64) {
        cudaFuncSetAttribute(dnc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dnc_kernel<0><<<(unsigned)grid, kThreadsD, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(dnc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dnc_kernel<1><<<(unsigned)grid, kThreadsD, smem, s>>>(a);
    }
    return cudaGetLastError();
}

// ------------------------------------------------- standalone linear advance
namespace {

template <int MODE>
__global__ void __launch_bounds__(kThreadsD) advance_kernel(const __grid_constant__ DncArgs a, const __grid_constant__ Params P0, int64_t count,
                                                            int64_t W, int64_t h, const double *in,
                                                            double *out)
{
    using V = typename fft::Cx<MODE>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ExpTables E;
    __shared__ SpecEntry cache[kSpecSlots];
    __shared__ int ncache;
    __shared__ int64_t arena_used;
    V *sm = (V *)smem_raw;
    char *slot = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    Counters cnt{0, 0, 0, 0, 0, 0, 0};
    if (threadIdx.x == 0) { ncache = 0; arena_used = 0; }
    __syncthreads();
    const int64_t nout = W - (int64_t)(P0.nw - 1) * h;
    for (int64_t s = blockIdx.x; s < count; s += gridDim.x) {
        Dnc<MODE> d(a, P0, E, sm, slot, cache, &ncache, &arena_used, nullptr, cnt);
        Buf bi{const_cast<double *>(in) + s * W, 0};
        Buf bo{out + s * nout, 0};
        d.conv(bi, 0, W - 1, bo, h);
    }
}

}  // namespace

size_t linear_advance_workspace_bytes(int method, int64_t W, int64_t h)
{
    (void)h;
    Layout L = make_layout(method, (W + 1) / 2 + 1, 16);
    return (size_t)(L.stride * 64 + 4096);
}

cudaError_t run_linear_advance(int method, int nw, const double *w, int64_t count, int64_t W, int64_t h,
                               const double *d_in, double *d_out, const void *d_tw, int tw_log2,
                               void *ws, size_t ws_bytes, int *d_err, cudaStream_t s)
{
    Layout L = make_layout(method, (W + 1) / 2 + 1, 16);
    int64_t grid = std::min<int64_t>(count, 64);
    if ((size_t)(grid * L.stride) > ws_bytes) grid = (int64_t)(ws_bytes / L.stride);
    if (grid < 1) return cudaErrorMemoryAllocation;
    if (tw_log2 < L.tw_log2) return cudaErrorInvalidValue;
    Params P;
    memset(&P, 0, sizeof(P));
    P.model = AOP_BINOMIAL_CALL;
    P.nw = nw;
    P.D = nw - 1;
    P.o_min = 0;
    P.w[0] = w[0]; P.w[1] = w[1]; P.w[2] = nw == 3 ? w[2] : 0.0;
    P.wsum = P.w[0] + P.w[1] + P.w[2];
    DncArgs a;
    memset(&a, 0, sizeof(a));
    a.B = 16;
    a.lg_nsmem = L.lg_nsmem;
    a.W_max = L.W_max;
    a.ws = (char *)ws;
    a.ws_stride = L.stride;
    a.off_r0 = L.off_r0; a.off_mid = L.off_mid; a.off_scr = L.off_scr; a.off_spec = L.off_spec;
    a.spec_cap = L.spec_cap;
    a.tw = d_tw;
    a.tw_log2 = tw_log2;
    a.err = d_err;
    const size_t smem = (size_t)((method == AOP_FFT_FP64) ? 16 : 8) << L.lg_nsmem;
    if (method == AOP_FFT_FP64) {
        cudaFuncSetAttribute(advance_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        advance_kernel<0><<<(unsigned)grid, kThreadsD, smem, s>>>(a, P, count, W, h, d_in, d_out);
    } else {
        cudaFuncSetAttribute(advance_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        advance_kernel<1><<<(unsigned)grid, kThreadsD, smem, s>>>(a, P, count, W, h, d_in, d_out);
    }
    return cudaGetLastError();
}

// ----------------------------------------------- allocation-free linear advance
// For callers that must not allocate device memory at call time (a serving
// thread that runs under a fixed memory budget, an embedding host whose
// allocator owns all device memory, code that cannot afford the implicit
// synchronisation of cudaMalloc/cudaFree).  The scratch space of the linear
// advance lives in one file-scope device array instead of a context
// workspace.  Every GPU that loads the library holds this array until the
// process exits.
namespace {

constexpr int64_t kNoAllocMaxW = AOP_NOALLOC_MAX_W;     // widest segment accepted
constexpr int64_t kNoAllocNmax = AOP_NOALLOC_MAX_W;     // largest transform length
constexpr int kNoAllocCtas = 16;
constexpr int kNoAllocTwLog2 = 15;                      // twiddles for N <= 2^15
constexpr int64_t kNoAllocSpec = kNoAllocNmax / 2 + 2;  // one kernel power per call
constexpr int64_t kNoAllocStride = kNoAllocNmax * 16 + kNoAllocSpec * 16;   // FP64 worst case
constexpr int64_t kNoAllocTwEntries = (int64_t)1 << (kNoAllocTwLog2 - 1);
constexpr int64_t kNoAllocTw32Off = kNoAllocCtas * kNoAllocStride;
constexpr int64_t kNoAllocTw64Off = kNoAllocTw32Off + kNoAllocTwEntries * 16;
constexpr int64_t kNoAllocBytes = kNoAllocTw64Off + kNoAllocTwEntries * 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// device address of the array, looked up once per device (host code may not
// use the array's name as a device pointer)
struct NoAllocDevice {
    bool ready;
    char *base;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

}  // namespace

}  // namespace aop

extern "C" aop_status aop_linear_advance_noalloc(int method, int nw, const double *w, int64_t count,
                                                 int64_t W, int64_t h, const double *d_in, double *d_out,
                                                 void *stream)
{
    using namespace aop;
    if (!w || (count > 0 && (!d_in || !d_out))) return AOP_EINVAL;
    if (method != AOP_FFT_FP64 && method != AOP_FFT_FP32SPLIT) return AOP_EINVAL;
    if (nw < 2 || nw > 3 || h < 1 || count < 0 || W < 2 || W > kNoAllocMaxW ||
        (int64_t)(nw - 1) * h >= W)
        return AOP_EINVAL;
    if (count == 0) return AOP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return AOP_ECUDA; }
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        NoAllocDevice &D = g_noalloc_dev[dev];
        if (!D.ready) {
            // one-time set-up on this device: find the array and fill the
            // twiddle tables it holds (nothing is allocated)
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) { cudaGetLastError(); return AOP_ECUDA; }
            char *b = (char *)ptr;
            e = launch_twiddles(kNoAllocTwLog2, b + kNoAllocTw32Off, b + kNoAllocTw64Off, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { cudaGetLastError(); return AOP_ECUDA; }
            D.base = b;
            D.ready = true;
        }
        base = D.base;
    }
    Params P;
    memset(&P, 0, sizeof(P));
    P.model = AOP_BINOMIAL_CALL;
    P.nw = nw;
    P.D = nw - 1;
    P.o_min = 0;
    P.w[0] = w[0]; P.w[1] = w[1]; P.w[2] = nw == 3 ? w[2] : 0.0;
    P.wsum = P.w[0] + P.w[1] + P.w[2];
    DncArgs a;
    memset(&a, 0, sizeof(a));
    a.B = 16;
    a.lg_nsmem = (method == AOP_FFT_FP64) ? 11 : 12;
    a.W_max = kNoAllocMaxW;
    a.ws = base;
    a.ws_stride = kNoAllocStride;
    a.off_scr = 0;
    a.off_spec = kNoAllocNmax * 16;
    a.spec_cap = kNoAllocSpec;
    a.tw = base + ((method == AOP_FFT_FP64) ? kNoAllocTw64Off : kNoAllocTw32Off);
    a.tw_log2 = kNoAllocTwLog2;
    a.err = nullptr;
    const int64_t grid = std::min<int64_t>(count, kNoAllocCtas);
    const size_t smem = (size_t)((method == AOP_FFT_FP64) ? 16 : 8) << a.lg_nsmem;
    if (method == AOP_FFT_FP64) {
        cudaFuncSetAttribute(advance_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        advance_kernel<0><<<(unsigned)grid, kThreadsD, smem, s>>>(a, P, count, W, h, d_in, d_out);
    } else {
        cudaFuncSetAttribute(advance_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        advance_kernel<1><<<(unsigned)grid, kThreadsD, smem, s>>>(a, P, count, W, h, d_in, d_out);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AOP_OK : AOP_ECUDA;
}
