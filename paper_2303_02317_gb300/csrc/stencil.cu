// stencil.cu -- the plain Theta(T^2) backward induction on the GPU (hot-path
// row a8): Fig. 1's nested loop for the binomial call and its analogues for the
// trinomial call (Sec. 3) and the BSM explicit scheme (Sec. 4, bsmG), with the
// early-exercise max at every cell.
//
// Layout: per option an exercise table ex[k'] (k' in [0, 2T]) and two row
// buffers (ping-pong) of D T + 1 (calls) or 2T + 1 (put) doubles, at a uniform
// stride.  One launch advances every option of the batch by up to kRows rows:
// each warp owns a tile of contiguous cells held in registers (kLC per lane),
// steps the rows there with shuffles between neighbouring lanes, and reads the
// exercise values from its slice of the table in shared memory (overlapped
// tiling: the cells a tile's rows cut off are recomputed by the neighbour
// tile).  The per-row divider is reduced per warp and merged with atomicMax.
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

constexpr int kRows = 32;       // rows per temporal block (one launch): 16 KB of exercise slices a warp, three CTAs per SM
constexpr int kLC = 16;         // cells per lane: a warp tile holds 32 x kLC contiguous cells
constexpr int kTile = 32 * kLC;
constexpr int kWarps = 4;       // warp tiles per CTA

// Each warp keeps a slice of the option's exercise table in shared memory,
// one segment per lane: lane l's segment holds the entries its cells read over
// the block's rows, at offsets alpha c + beta (k - 1) (cell c of the lane, row
// k of the block; alpha = 2 on the binomial lattice, 1 else; beta = 1 for the
// calls, whose exercise value moves one exponent per row, 0 for the put).  The
// segment length is odd, so the 32 lanes' reads fall in distinct banks, and a
// cell's address is a per-row base plus a constant.
__host__ __device__ constexpr int seg_vmax(int alpha, int beta) { return alpha * (kLC - 1) + beta * (kRows - 1); }
__host__ __device__ constexpr int seg_stride(int alpha, int beta) { return (seg_vmax(alpha, beta) + 1) | 1; }
constexpr int kSegMax = seg_stride(2, 1) > seg_stride(1, 1) ? seg_stride(2, 1) : seg_stride(1, 1);
constexpr size_t kWarpTab = (size_t)32 * kSegMax * sizeof(double);

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

// One temporal block of up to kRows rows of every option (grid.y walks the
// options, grid.x x kWarps the warp tiles of an option's output row).  A warp
// loads its input window of kTile cells (lane l: cells x0 + kLC l .. + kLC-1),
// steps the rows in registers -- the D cells right of a lane's last cell (and
// for the put the one left of its first) come from the neighbouring lanes by
// shuffle -- and stores the cells it owns.  The window's valid part shrinks by
// D cells per row on the right (calls) or one on each side (put); neighbouring
// tiles overlap by that much and compute the overlap identically.  Every cell
// takes max(continuation, exercise) (Def. 2.1); with BND each row's divider
// (calls: last red cell; put: last green cell) is reduced per warp and merged
// with atomicMax.
template <class C> struct Cell;
template <> struct Cell<double> {
    __device__ static double zero() { return 0.0; }
    __device__ static double shfl_dn(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
    __device__ static double shfl_up(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
    __device__ static double dot2(double w0, double w1, float2, float2, double a, double b) { return w0 * a + w1 * b; }
    __device__ static double dot3(double w0, double w1, double w2, float2, float2, float2, double a, double b,
                                  double c) { return w0 * a + w1 * b + w2 * c; }
    __device__ static bool ge(double a, double b) { return a >= b; }
    __device__ static bool clamped(double) { return false; }
};
template <> struct Cell<float2> {
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ static float2 shfl_dn(float2 v) {
        return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
    }
    __device__ static float2 shfl_up(float2 v) {
        return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
    }
    __device__ static float2 dot2(double, double, float2 v0, float2 v1, float2 a, float2 b) {
        return fft::df_dot2(v0, v1, a, b);
    }
    __device__ static float2 dot3(double, double, double, float2 v0, float2 v1, float2 v2, float2 a, float2 b,
                                  float2 c) { return fft::df_dot3(v0, v1, v2, a, b, c); }
    __device__ static bool ge(float2 a, float2 b) { return fft::df_ge(a, b); }
    __device__ static bool clamped(float2 e) { return e.x >= (float)kDfClamp; }
};

struct TileJob {
    int64_t T, R;        // steps of the option, rows left before this block
    int Kp;              // rows of this block
    int64_t x0;          // first input cell of the warp's window
    int64_t own_lo, own_hi;
};

// the warp's table segments: lane l's entry v = table index kp_lo + alpha kLC l + v
template <class C>
__device__ void fill_tab(C *tab, const C *ex, int64_t kp_lo, int64_t T, int alpha, int vmax, int stride, int lane) {
    for (int l = 0; l < 32; l++) {
        const int64_t b = kp_lo + (int64_t)alpha * kLC * l;
        for (int v = lane; v <= vmax; v += 32) {
            const int64_t kp = min(max(b + v, (int64_t)0), 2 * T);
            tab[l * stride + v] = ex[kp];
        }
    }
    __syncwarp();
}

// Calls: input row R (columns 0 .. D R), rows R-1 .. R-Kp.
template <class C, int D, bool BND>
__device__ long long call_tile(const Params &P, const TileJob &J, const C *src, C *dst, const C *ex, C *tab,
                               int32_t *b, int lane) {
    using A = Cell<C>;
    const int alpha = (D == 1) ? 2 : 1;
    const int stride = seg_stride(alpha, 1);
    const int64_t R = J.R, x0 = J.x0;
    const int64_t xl = x0 + (int64_t)kLC * lane;              // the lane's first cell
    fill_tab(tab, ex, ex_index(P, R - 1, x0), J.T, alpha, seg_vmax(alpha, 1), stride, lane);
    C v[kLC + 2];
#pragma unroll
    for (int c = 0; c < kLC; c++) {
        const int64_t x = xl + c;
        v[c] = (x >= 0 && x <= (int64_t)D * R) ? src[x] : A::zero();
    }
    const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
    const float2 f0 = fft::df_from(w0), f1 = fft::df_from(w1), f2 = fft::df_from(w2);
    const C *tl = tab + lane * stride;
    long long cells = 0;
    for (int k = 1; k <= J.Kp; k++) {
        v[kLC] = A::shfl_dn(v[0]);
        if (D == 2) v[kLC + 1] = A::shfl_dn(v[1]);
        const C *tk = tl + (k - 1);
        const int64_t hi = min(x0 + kTile - 1 - (int64_t)D * k, (int64_t)D * (R - k));   // last valid cell
        const int lim = (int)max(min(hi - xl, (int64_t)kLC - 1), (int64_t)-1);
        int last = -1;
#pragma unroll
        for (int c = 0; c < kLC; c++) {
            const C cont = (D == 2) ? A::dot3(w0, w1, w2, f0, f1, f2, v[c], v[c + 1], v[c + 2])
                                    : A::dot2(w0, w1, f0, f1, v[c], v[c + 1]);
            const C e = tk[alpha * c];
            const bool red = A::ge(cont, e) && !A::clamped(e);
            v[c] = red ? cont : e;
            if (BND && red && c <= lim) last = c;
        }
        if (BND) {
            int best = (last >= 0) ? (int)(xl + last) : INT32_MIN;
            best = __reduce_max_sync(0xffffffffu, best);
            if (lane == 0 && best != INT32_MIN) atomicMax(&b[R - k], best);
        }
        cells += max(hi - x0 + 1, (int64_t)0);
    }
#pragma unroll
    for (int c = 0; c < kLC; c++) {
        const int64_t x = xl + c;
        if (x >= J.own_lo && x <= J.own_hi) dst[x] = v[c];
    }
    return cells;
}

// BSM put: input row n0 = T - R (k in [-R, R], stored at k + T), rows n0+1 ..
// n0+Kp; weights b, c, a on k-1, k, k+1; the exercise value does not depend on
// the row.
template <class C, bool BND>
__device__ long long put_tile(const Params &P, const TileJob &J, const C *src, C *dst, const C *ex, C *tab,
                              int32_t *b, int lane) {
    using A = Cell<C>;
    const int stride = seg_stride(1, 0);
    const int64_t R = J.R, x0 = J.x0, T = J.T;
    const int64_t xl = x0 + (int64_t)kLC * lane;
    fill_tab(tab, ex, x0 + T, T, 1, seg_vmax(1, 0), stride, lane);
    C v[kLC];
#pragma unroll
    for (int c = 0; c < kLC; c++) {
        const int64_t x = xl + c;
        v[c] = (x >= -R && x <= R) ? src[x + T] : A::zero();
    }
    const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
    const float2 f0 = fft::df_from(w0), f1 = fft::df_from(w1), f2 = fft::df_from(w2);
    const C *tl = tab + lane * stride;
    const int64_t n0 = T - R;
    long long cells = 0;
    for (int k = 1; k <= J.Kp; k++) {
        const C left = A::shfl_up(v[kLC - 1]);
        const C right = A::shfl_dn(v[0]);
        const int64_t lo = max(x0 + k, -(R - k)), hi = min(x0 + kTile - 1 - k, R - k);   // valid cells
        const int clo = (int)max(min(lo - xl, (int64_t)kLC), (int64_t)0);
        const int chi = (int)max(min(hi - xl, (int64_t)kLC - 1), (int64_t)-1);
        int last = -1;
        C prev = left;
#pragma unroll
        for (int c = 0; c < kLC; c++) {
            const C nxt = (c + 1 < kLC) ? v[(c + 1) % kLC] : right;
            const C cont = A::dot3(w0, w1, w2, f0, f1, f2, prev, v[c], nxt);
            const C e = tl[c];
            const bool green = !A::ge(cont, e);
            prev = v[c];
            v[c] = green ? e : cont;
            if (BND && green && c >= clo && c <= chi) last = c;
        }
        if (BND) {
            int best = (last >= 0) ? (int)(xl + last) : INT32_MIN;
            best = __reduce_max_sync(0xffffffffu, best);
            if (lane == 0 && best != INT32_MIN) atomicMax(&b[n0 + k], best);
        }
        cells += max(hi - lo + 1, (int64_t)0);
    }
#pragma unroll
    for (int c = 0; c < kLC; c++) {
        const int64_t x = xl + c;
        if (x >= J.own_lo && x <= J.own_hi) dst[x + T] = v[c];
    }
    return cells;
}

// output cells a warp tile owns: the window less what its rows cut off
__host__ __device__ inline int tile_out(int D, bool put) { return kTile - (put ? 2 : D) * kRows; }

template <bool DF, bool BND>
__global__ void __launch_bounds__(kWarps * 32)
stencil_tile_kernel(const Params *params, int64_t n, int64_t T_max, int64_t launch, double *ws, int32_t *bnd,
                    const int64_t *bnd_off, long long *cells)
{
    using C = typename std::conditional<DF, float2, double>::type;   // one 8-byte cell
    static_assert(sizeof(C) == sizeof(double), "cells share the FP64 layout");
    extern __shared__ __align__(16) double tab_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *tab = (C *)(tab_raw + (size_t)warp * 32 * kSegMax);
    const StencilOpt L = stencil_layout(T_max);
    long long my_cells = 0;
    for (int64_t o = blockIdx.y; o < n; o += gridDim.y) {
        const Params &P = params[o];
        if (P.status != AOP_OK) continue;
        const bool put = (P.model == AOP_BSM_PUT);
        TileJob J;
        J.T = P.T;
        J.R = J.T - launch * (int64_t)kRows;
        if (J.R <= 0) continue;
        J.Kp = (int)min((int64_t)kRows, J.R);
        const int64_t Rout = J.R - J.Kp;
        const int D = P.D;
        const int64_t out_lo = put ? -Rout : 0, out_hi = put ? Rout : (int64_t)D * Rout;
        const int outw = tile_out(D, put);
        const int64_t ntiles = (out_hi - out_lo + outw) / outw;
        const int64_t tile = (int64_t)blockIdx.x * kWarps + warp;
        if (tile >= ntiles) continue;
        J.own_lo = out_lo + tile * outw;
        J.own_hi = min(J.own_lo + outw - 1, out_hi);
        J.x0 = put ? J.own_lo - J.Kp : J.own_lo;
        const C *ex = (const C *)(ws + o * L.stride);
        const C *rowA = (const C *)(ws + o * L.stride + L.W);
        const C *src = (launch % 2 == 0) ? rowA : rowA + L.W;
        C *dst = (C *)((launch % 2 == 0) ? rowA + L.W : rowA);
        int32_t *b = bnd ? bnd + bnd_off[o] : nullptr;
        if (put) my_cells += put_tile<C, BND>(P, J, src, dst, ex, tab, b, lane);
        else if (D == 2) my_cells += call_tile<C, 2, BND>(P, J, src, dst, ex, tab, b, lane);
        else my_cells += call_tile<C, 1, BND>(P, J, src, dst, ex, tab, b, lane);
        __syncwarp();
    }
    if (cells && lane == 0 && my_cells) atomicAdd((unsigned long long *)cells, (unsigned long long)my_cells);
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
    const int64_t launches = (T_max + kRows - 1) / kRows;
    long long *cells = d_stats ? (long long *)&d_stats->stencil_cells : nullptr;
    // warp tiles of the widest output row (the narrowest tile: 3-point stencils)
    const int64_t max_tiles = (2 * T_max + 1 + tile_out(2, true) - 1) / tile_out(2, true);
    const dim3 grid((unsigned)((max_tiles + kWarps - 1) / kWarps), (unsigned)std::min<int64_t>(n, 65535));
    const size_t smem = kWarps * kWarpTab;
    auto kern = d_bnd ? stencil_tile_kernel<DF, true> : stencil_tile_kernel<DF, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int64_t l = 0; l < launches; l++)
        kern<<<grid, kWarps * 32, smem, s>>>(d_params, n, T_max, l, w, d_bnd, d_bnd_off, cells);
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
