// stencil.cu -- the plain Theta(T^2) backward induction on the GPU (hot-path
// row a8): Fig. 1's nested loop for the binomial call and its analogues for the
// trinomial call (Sec. 3) and the BSM explicit scheme (Sec. 4, bsmG), with the
// early-exercise max at every cell.
//
// Layout: per option an exercise table ex[k'] (k' in [0, 2T]) and two row
// buffers (ping-pong) of D T + 1 (calls) or 2T + 1 (put) doubles, at a uniform
// stride.  One launch advances every option of the batch by up to kRows rows:
// a CTA owns an output segment of kSeg cells, loads the input row segment plus
// the halo its dependency cone needs (kRows*D cells to the right for the calls,
// kRows on each side for the put) into shared memory, and steps kRows rows
// there (overlapped tiling: the halo is recomputed by the neighbour tile).
// The per-row divider is reduced per tile and merged with atomicMax.
//
// Two arithmetics (template flag DF): FP64, and doubled FP32 (a cell is an
// unevaluated pair hi + lo of FP32 numbers in the same 8-byte slot, ~48-bit
// significands, summed on the FP32 pipe).  On this GPU an FP64 warp
// instruction occupies a sub-partition's FP64 unit for ~64 cycles, so the
// doubled-FP32 loop is the faster plain form; its values carry ~2^-48 relative
// rounding per row.  Doubled-FP32 exercise values are clamped to +-1e30 (FP32
// range).  The clamp lies at least ln(1e28) = 64 log-price units from any node
// within e^2 of the spot or strike, many standard deviations of the walk
// (sigma sqrt(expiry) < 2 for every supported request), so its effect on the
// root value is below the rounding: the clamped cells only meet the root
// through transition weights far under 1e-300.  Call cells at the clamp are
// taken as green (as the D&C does for node prices past its range): they lie far
// above every early-exercise boundary with a yield, and without one (whole rows
// red) the reported divider stops below the clamp.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace aop {

namespace {

constexpr int kRows = 128;      // rows per temporal block (one launch)
constexpr int kSeg = 2048;      // output cells per tile
constexpr int kThreads = 256;
constexpr int kBuf = kSeg + 2 * kRows + 8;

struct StencilOpt {
    int64_t W;        // row buffer length (doubles)
    int64_t stride;   // doubles per option in the workspace
};

__host__ __device__ inline StencilOpt stencil_layout(int64_t T_max) {
    StencilOpt L;
    L.W = 2 * T_max + 1;                   // enough for every model
    L.stride = ((3 * L.W + 31) / 32) * 32; // ex table + two rows
    return L;
}

__device__ inline int64_t remaining_after(int64_t T, int64_t launch) {
    int64_t r = T - launch * (int64_t)kRows;
    return r < 0 ? 0 : r;
}

constexpr double kDfClamp = 1e30;

// a cell value as stored by the arithmetic DF (FP64, or the pair hi, lo)
template <bool DF>
__device__ __forceinline__ void put_cell(double *p, double v) {
    if (DF) *(float2 *)p = fft::df_from(fmin(fmax(v, -kDfClamp), kDfClamp));
    else *p = v;
}

// Exercise table and the first row (calls: row T; put: row 0), and the divider
// of that row.  grid: (chunks, n).
template <bool DF>
__global__ void stencil_init_kernel(const Params *params, int64_t n, int64_t T_max, double *ws,
                                    int32_t *bnd, const int64_t *bnd_off)
{
    __shared__ ExpTables E;
    for (int64_t o = blockIdx.y; o < n; o += gridDim.y) {
    const Params P = params[o];
    if (P.status != AOP_OK) continue;
    __syncthreads();
    build_exp_tables(P, E);
    __syncthreads();
    const StencilOpt L = stencil_layout(T_max);
    double *ex = ws + o * L.stride;
    double *row = ex + L.W;
    const int64_t T = P.T;
    int best = (P.model == AOP_BSM_PUT) ? INT32_MIN : -1;
    for (int64_t kp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kp <= 2 * T;
         kp += (int64_t)gridDim.x * blockDim.x) {
        double e = exercise(P, E, kp);
        put_cell<DF>(&ex[kp], e);
        if (P.model == AOP_BSM_PUT) {
            // row 0 holds k in [-T, T] at index k + T = kp; continuation 0
            put_cell<DF>(&row[kp], e > 0.0 ? e : 0.0);
            if (e > 0.0) best = max(best, (int)(kp - T));
        } else {
            // row T: column j has k' = 2j (binomial) or j (trinomial)
            int64_t j;
            bool hit;
            if (P.model == AOP_BINOMIAL_CALL) { hit = (kp % 2 == 0); j = kp / 2; }
            else { hit = true; j = kp; }
            if (hit) {
                put_cell<DF>(&row[j], e > 0.0 ? e : 0.0);
                if (0.0 >= e) best = max(best, (int)j);
            }
        }
    }
    if (bnd) {
        int32_t *b = bnd + bnd_off[o];
        int64_t top = (P.model == AOP_BSM_PUT) ? 0 : T;
        // initialise every row's divider to "none", then merge the top row
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= T;
             r += (int64_t)gridDim.x * blockDim.x)
            if (r != top) b[r] = (P.model == AOP_BSM_PUT) ? INT32_MIN : -1;
        // the top row's entry was set to "none" by top_boundary_kernel, which
        // runs earlier on the same stream; every block merges into it.
        best = __reduce_max_sync(0xffffffffu, best);
        if ((threadIdx.x & 31) == 0) atomicMax(&b[top], best);
    }
    }
}

// One temporal block of up to kRows rows for every option.  grid-stride over
// tiles; tile -> (option, segment) through per-option tile counts computed in
// shared memory.
template <bool DF>
__global__ void __launch_bounds__(kThreads)
stencil_block_kernel(const Params *params, int64_t n, int64_t T_max, int64_t launch,
                     double *ws, int32_t *bnd, const int64_t *bnd_off, long long *cells)
{
    using C = typename std::conditional<DF, float2, double>::type;   // one 8-byte cell
    static_assert(sizeof(C) == sizeof(double), "cells share the FP64 layout");
    __shared__ double buf_raw[2][kBuf];
    C (*buf)[kBuf] = (C (*)[kBuf])buf_raw;
    __shared__ int s_bnd[kRows + 1];
    __shared__ int64_t s_tiles_total;
    const StencilOpt L = stencil_layout(T_max);

    // count tiles of all options (n is modest for this path; every block redoes it)
    if (threadIdx.x == 0) {
        int64_t tot = 0;
        for (int64_t o = 0; o < n; o++) {
            const Params &P = params[o];
            if (P.status != AOP_OK) continue;
            int64_t R = remaining_after(P.T, launch);
            if (R == 0) continue;
            int64_t Rout = R - min((int64_t)kRows, R);
            int64_t width = (P.model == AOP_BSM_PUT) ? 2 * Rout + 1 : (int64_t)P.D * Rout + 1;
            tot += (width + kSeg - 1) / kSeg;
        }
        s_tiles_total = tot;
    }
    __syncthreads();
    const int64_t total = s_tiles_total;
    long long my_cells = 0;

    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        // locate option and segment (linear scan; n is small for this path)
        int64_t o = 0, seg = t;
        for (o = 0; o < n; o++) {
            const Params &P = params[o];
            if (P.status != AOP_OK) continue;
            int64_t R = remaining_after(P.T, launch);
            if (R == 0) continue;
            int64_t Rout = R - min((int64_t)kRows, R);
            int64_t width = (P.model == AOP_BSM_PUT) ? 2 * Rout + 1 : (int64_t)P.D * Rout + 1;
            int64_t nt = (width + kSeg - 1) / kSeg;
            if (seg < nt) break;
            seg -= nt;
        }
        const Params P = params[o];
        const int64_t T = P.T;
        const int64_t R = remaining_after(T, launch);
        const int Kp = (int)min((int64_t)kRows, R);
        const int64_t Rout = R - Kp;
        const C *ex = (const C *)(ws + o * L.stride);
        C *rowA = (C *)(ws + o * L.stride + L.W);
        C *rowB = rowA + L.W;
        const C *src = (launch % 2 == 0) ? rowA : rowB;
        C *dst = (launch % 2 == 0) ? rowB : rowA;
        const bool put = (P.model == AOP_BSM_PUT);
        const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        const float2 v0 = fft::df_from(w0), v1 = fft::df_from(w1), v2 = fft::df_from(w2);
        const int nw = P.nw;
        const int64_t nseg = ((put ? 2 * Rout + 1 : (int64_t)P.D * Rout + 1) + kSeg - 1) / kSeg;

        // absolute coordinates: calls use column j (row r holds [0, D r]);
        // the put uses k (row n holds [-(T-n), T-n]) and stores at k + T.
        int64_t a0, in_lo, in_hi;      // output segment start, input window
        if (!put) {
            a0 = seg * kSeg;
            in_lo = a0;
            in_hi = min(a0 + kSeg - 1 + (int64_t)P.D * Kp, (int64_t)P.D * R);
        } else {
            a0 = -Rout + seg * kSeg;
            in_lo = max(a0 - Kp, -R);
            in_hi = min(a0 + kSeg - 1 + Kp, R);
        }
        const int64_t base = in_lo;
        const int64_t own_lo = (seg == 0) ? INT64_MIN / 2 : a0;
        const int64_t own_hi = (seg == nseg - 1) ? INT64_MAX / 2 : a0 + kSeg - 1;
        const int64_t store_off = put ? T : 0;

        for (int64_t x = in_lo + threadIdx.x; x <= in_hi; x += blockDim.x)
            buf[0][x - base] = src[x + store_off];
        for (int k = threadIdx.x; k <= Kp; k += blockDim.x) s_bnd[k] = INT32_MIN;
        __syncthreads();

        int cur = 0;
        int64_t lo = in_lo, hi = in_hi;
        for (int k = 1; k <= Kp; k++) {
            // row index of the new row: calls r = R - k; put n = T - R + k
            const int64_t r = put ? (T - R + k) : (R - k);
            int64_t nlo, nhi;
            if (!put) { nlo = lo; nhi = min(hi - P.D, (int64_t)P.D * r); }
            else { nlo = max(lo + 1, -(T - r)); nhi = min(hi - 1, T - r); }
            const C *pv = buf[cur];
            C *nv = buf[cur ^ 1];
            int best = INT32_MIN;
            for (int64_t x = nlo + threadIdx.x; x <= nhi; x += blockDim.x) {
                const int64_t ix = x - base;
                C cont;
                if constexpr (DF) {
                    if (!put) cont = (nw == 3) ? fft::df_dot3(v0, v1, v2, pv[ix], pv[ix + 1], pv[ix + 2])
                                               : fft::df_dot2(v0, v1, pv[ix], pv[ix + 1]);
                    else cont = fft::df_dot3(v0, v1, v2, pv[ix - 1], pv[ix], pv[ix + 1]);
                } else {
                    if (!put) {
                        cont = w0 * pv[ix] + w1 * pv[ix + 1];
                        if (nw == 3) cont += w2 * pv[ix + 2];
                    } else {
                        cont = w0 * pv[ix - 1] + w1 * pv[ix] + w2 * pv[ix + 1];
                    }
                }
                const C e = ex[ex_index(P, r, x)];
                bool ge;
                if constexpr (DF) ge = fft::df_ge(cont, e);
                else ge = cont >= e;
                bool take_ex;
                if (!put) {
                    bool red = ge;
                    if constexpr (DF) red = red && e.x < (float)kDfClamp;
                    take_ex = !red;
                    if (red && x >= own_lo && x <= own_hi) best = max(best, (int)x);
                } else {
                    take_ex = !ge;
                    if (take_ex && x >= own_lo && x <= own_hi) best = max(best, (int)x);
                }
                nv[ix] = take_ex ? e : cont;
                my_cells++;
            }
            best = __reduce_max_sync(0xffffffffu, best);
            if ((threadIdx.x & 31) == 0 && best != INT32_MIN) atomicMax(&s_bnd[k], best);
            lo = nlo; hi = nhi;
            cur ^= 1;
            __syncthreads();
        }
        // write the owned output segment
        const int64_t out_hi = put ? min(a0 + kSeg - 1, Rout) : min(a0 + kSeg - 1, (int64_t)P.D * Rout);
        for (int64_t x = a0 + threadIdx.x; x <= out_hi; x += blockDim.x)
            dst[x + store_off] = buf[cur][x - base];
        if (bnd) {
            int32_t *b = bnd + bnd_off[o];
            for (int k = 1 + threadIdx.x; k <= Kp; k += blockDim.x) {
                const int64_t r = put ? (T - R + k) : (R - k);
                if (s_bnd[k] != INT32_MIN) atomicMax(&b[r], s_bnd[k]);
            }
        }
        __syncthreads();
    }
    if (cells) {
        my_cells = __reduce_add_sync(0xffffffffu, (unsigned)my_cells);
        if ((threadIdx.x & 31) == 0) atomicAdd((unsigned long long *)cells, (unsigned long long)my_cells);
    }
}

template <bool DF>
__global__ void stencil_finish_kernel(const Params *params, int64_t n, int64_t T_max, const double *ws,
                                      double *prices)
{
    const StencilOpt L = stencil_layout(T_max);
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const Params P = params[o];
        if (P.status != AOP_OK) { prices[o] = __longlong_as_double(0x7ff8000000000000ll); continue; }
        const int64_t launches = (P.T + kRows - 1) / kRows;
        const double *rowA = ws + o * L.stride + L.W;
        const double *row = (launches % 2 == 0) ? rowA : rowA + L.W;
        const int64_t at = (P.model == AOP_BSM_PUT) ? P.T : 0;
        double v;
        if (DF) {
            const float2 c = ((const float2 *)row)[at];
            v = (double)c.x + (double)c.y;
        } else {
            v = row[at];
        }
        prices[o] = v * P.out_scale;
    }
}

__global__ void top_boundary_kernel(const Params *params, int64_t n, int32_t *bnd, const int64_t *bnd_off)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const Params P = params[o];
        if (P.status != AOP_OK) continue;
        int64_t top = (P.model == AOP_BSM_PUT) ? 0 : P.T;
        bnd[bnd_off[o] + top] = (P.model == AOP_BSM_PUT) ? INT32_MIN : -1;
    }
}

}  // namespace

size_t stencil_workspace_bytes(int64_t n, int64_t T_max) {
    return (size_t)n * (size_t)stencil_layout(T_max).stride * sizeof(double) + 256;
}

template <bool DF>
static cudaError_t run_stencil_t(int64_t n, const Params *d_params, int64_t T_max, void *ws,
                                 double *d_prices, int32_t *d_status, int32_t *d_bnd,
                                 const int64_t *d_bnd_off, aop_stats *d_stats, cudaStream_t s)
{
    (void)d_status;          // statuses come from the parameter kernel
    if (n == 0) return cudaSuccess;
    double *w = (double *)ws;
    if (d_bnd) {
        top_boundary_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d_params, n, d_bnd, d_bnd_off);
    }
    {
        int chunks = (int)std::min<int64_t>((2 * T_max + 1 + 255) / 256, 1024);
        dim3 grid(chunks, (unsigned)std::min<int64_t>(n, 65535));
        stencil_init_kernel<DF><<<grid, 256, 0, s>>>(d_params, n, T_max, w, d_bnd, d_bnd_off);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t launches = (T_max + kRows - 1) / kRows;
    long long *cells = d_stats ? (long long *)&d_stats->stencil_cells : nullptr;
    for (int64_t l = 0; l < launches; l++) {
        stencil_block_kernel<DF><<<sms * 4, kThreads, 0, s>>>(d_params, n, T_max, l, w, d_bnd, d_bnd_off, cells);
    }
    stencil_finish_kernel<DF><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d_params, n, T_max, w, d_prices);
    return cudaGetLastError();
}

cudaError_t run_stencil(int64_t n, const Params *d_params, int64_t T_max, void *ws,
                        double *d_prices, int32_t *d_status, int32_t *d_bnd,
                        const int64_t *d_bnd_off, aop_stats *d_stats, cudaStream_t s, bool df)
{
    return df ? run_stencil_t<true>(n, d_params, T_max, ws, d_prices, d_status, d_bnd, d_bnd_off, d_stats, s)
              : run_stencil_t<false>(n, d_params, T_max, ws, d_prices, d_status, d_bnd, d_bnd_off, d_stats, s);
}

}  // namespace aop
