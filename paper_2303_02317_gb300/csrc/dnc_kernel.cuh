// dnc_kernel.cuh -- the trapezoidal divide-and-conquer pricer (hot-path rows a2-a7):
// its device code, compiled by dnc.cu (plain kernels, host side) and
// dnc_help.cu (the helping kernels).
//
// One CTA prices one option at a time (persistent grid over a device queue of
// options).  The recursion:
//
//   calls (binomial Sec. 2.3, trinomial appendix "Algorithm for American call
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
//   put (Sec. 4.3): green cells are left of the divider f, red cells right of
//   it.  region(n, lo, hi, f, h) advances the window [lo, hi] of row n to
//   [lo+h, hi-h] of row n+h in two halves; each half recurses on the
//   sub-trapezoid of base [f-2g, f+2g] around the divider ("trapezoid eglj"),
//   computes the red cells right of it with one FFT advance ("trapezoid fbnl")
//   and evaluates the green cells left of it in closed form.  The triangle is a
//   chain of trapezoids of halving height.
//
// Execution inside the CTA follows the paper's observation that each FFT
// advance can run in parallel with the recursion beside it (proof of Thm 2.8):
// one warp (the walker: in the FP32 modes the one on SM sub-partition 0, so that
// the walkers of an SM share it) runs the recursion and the base cases and posts
// every linear advance as a task in a per-depth slot; the other three warps
// (workers) execute the tasks (warp-level FFT convolutions) while the walker
// continues down the sub-trapezoid, and the walker waits for a task only when
// its output is needed.  The kernel power s(theta)^h of every (height, transform
// length) pair is evaluated once per option in FP64 on the band where |s|^h
// exceeds 2^-60 of its peak and cached.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

#include <type_traits>

namespace aop {

// Arguments of one pricing launch (shared by the translation units that
// compile the kernels).
struct DncArgs {
    const Params *params;
    int64_t n;
    int64_t grid;          // CTAs of the launch (boards to scan)
    int help_lg;           // advances with log2 N >= help_lg go on the board (0: no helping)
    int64_t off_board;     // byte offset of the CTA's board inside its slot
    int *finished;         // options finished so far (helpers stop at n)
    int help_block;        // helping CTAs run each board advance with all their warps
    unsigned epoch;        // this launch's stamp on board generations (stale boards are skipped)
    int B;                 // base-case height (2 .. 64 rows)
    int Bput;              // base-case height of the BSM put (its windows are four heights wide)
    int lg_tile;           // log2 of a worker's shared-memory transform tile
    int radix2;            // 1: transform stages as radix-2 steps only (else radix 4)
    int lg_block;          // log2 of the block-level tile (linear advance entry points)
    int64_t W_max;         // widest row (doubles)
    char *ws;
    int64_t ws_stride;     // bytes per CTA
    int64_t off_r0, off_mid, off_scr, off_spec;   // byte offsets inside a CTA slot
    int64_t scr_stride;    // bytes of global transform scratch per worker
    int64_t mid_off[kMaxDepth];                   // doubles, relative to off_mid
    int64_t spec_cap;      // arena entries
    const void *tw;
    int tw_log2;
    double *prices;
    int32_t *status;
    int32_t *bnd;
    const int64_t *bnd_off;
    int *queue;
    int *sm_slots;         // per-SM arrival counters (1024 ints, zeroed per launch)
    int *err;
    aop_stats *stats;
    int64_t *opt_ns;       // per-option device time (nullable)
    double *greeks;        // per option delta, gamma, theta (nullable)
    int flags;             // AOP_FLAG_* bits
    const int32_t *order;  // batch: the i-th option taken is order[i] (nullable: i)
    // serving session (sreq == nullptr in batch mode): requests are read from
    // host memory as the host publishes them; prices, status and a done flag
    // go back to host memory per request
    const aop_request *sreq;
    const volatile long long *spub;    // requests published so far
    const volatile int *sstop;         // the host asks the kernel to exit
    unsigned long long *sclaim;        // requests claimed so far (device memory)
    volatile int32_t *sdone;           // 1 once request o's result is written
    int64_t sT_max;                    // longest T the session's workspace holds
};

// Launch the helping pricing kernel of a method (dnc_help.cu); the dynamic
// shared memory attribute is set here.
cudaError_t launch_dnc_help(int method, unsigned grid, int threads, size_t smem, cudaStream_t s,
                            const DncArgs &a);

namespace {

// CTA shape: one walker warp plus three worker warps.  Workers below `big`
// may take multi-pass transforms (each owns a global scratch area; all three
// do: a long advance never waits for one of two scratch owners).  Seven
// workers per option (two options per SM) lost to this shape in the
// doubled-FP32 mode: shorter waits, but slower base cases.  min_ctas sets the
// register budget: 128 a thread for four options per SM (FP32-split), 255 for
// two (doubled FP32 and FP64, whose transforms need the registers and whose
// best schedules keep two options per SM).
template <int MODE> struct Shape {
    static constexpr int warps = 4;
    static constexpr int threads = 32 * warps;
    static constexpr int workers = warps - 1;
    static constexpr int big = 3;
    static constexpr int min_ctas = (MODE == 1) ? 4 : 2;
};
inline int shape_workers(int) { return Shape<0>::workers; }
inline int shape_big(int) { return Shape<0>::big; }
constexpr int kThreadsA = 128;             // linear-advance entry points (block-level transforms)
constexpr int kSpecSlots = 128;
constexpr int kSpecLg = 22;                // log2 g and log2 N of directly indexed spectra
constexpr int kLeftoverCall = 48;          // rows solved naively at the root
constexpr double kDfLogRange = 80.0;       // largest log price ratio of a doubled-FP32 base case
constexpr int kRegCells = 256;             // widest base-case window: 8 registers per lane
constexpr int kNaiveCap = 640;             // exercise table of a base case: a 256-cell binomial
                                           // window over 64 rows spans 2 x 256 + 64 + 4 exponents
constexpr uint64_t kWaitNs = 30ull * 1000000000ull;   // bound of every spin-wait (30 s)
constexpr uint64_t kHelpIdleNs = 20000000ull;          // a helping CTA without work for 20 ms stops
constexpr uint64_t kHelpDeferNs = 50000ull;             // own workers leave board tasks to helpers this long
constexpr int kGenBits = 28;                           // board generation: launch epoch << kGenBits | count
constexpr uint64_t kStallNs = 20000000ull;             // the bound under AOP_FLAG_TEST_STALL (20 ms)

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

enum { TASK_FREE = 0, TASK_POSTED = 1, TASK_CLAIMED = 2, TASK_DONE = 3,
       TASK_BOARD = 4 };     // (local slot only) the task of this depth sits on the CTA's board
enum { SPEC_BUILDING = 1, SPEC_READY = 2 };

struct SpecEntry {
    int32_t g;
    int32_t lgN;
    int32_t mc;
    volatile int32_t state;
    int64_t off;
    int64_t n0;           // tilted advances: output factor e^{-kappa (n - n0)} resid
    float2 resid;
    double resid64;
};

// Per-advance output scaling: 1/N (FP64 and FP32 copies, both exact powers
// of two) and the tilt's output factor.
struct ConvScale {
    double d;
    float f;
    int64_t n0;
    float2 resid;
    double resid64;
};

// e^{g tL - kappa n0} with n0 = floor(g tL / kappa): the part of a g-step
// tilted advance's output factor e^{g tL - kappa n} left after the table
// factor e^{-kappa (n - n0)}; n >= D g > n0 for every output cell.
__device__ inline void tilt_shift(const Params &P, int64_t g, int64_t &n0, float2 &resid, double &resid64) {
    const double e = (double)g * P.tL;
    const double q = floor(e / P.kappa);
    n0 = (int64_t)q;
    const double v = exp(e - P.kappa * q);
    const float h = (float)v;
    resid = make_float2(h, (float)(v - (double)h));
    resid64 = v;
}

// a row segment in memory: the value of column x lives at p[x - base]
struct Buf {
    double *p;
    int64_t base;
};

// Row values as the pricer stores them (FP64 in mode 0, FP32 pairs hi + lo
// otherwise), read and written in FP64 by the base cases and first rows.
template <int MODE>
__device__ __forceinline__ double cell_ld(const Buf &b, int64_t x) {
    return fft::cell_value(((const typename fft::CellT<MODE>::T *)b.p)[x - b.base]);
}
template <int MODE>
__device__ __forceinline__ void cell_st(const Buf &b, int64_t x, double v) {
    ((typename fft::CellT<MODE>::T *)b.p)[x - b.base] = fft::make_cell<MODE>(v);
}

struct Task {
    Buf in, out;
    int64_t x_lo, x_hi, g;
    int32_t lgN;
    volatile int32_t state;
};

// Helping (batch launches).  An option's multi-pass advances (transform
// larger than a worker tile) are posted on its CTA's board in global memory.
// The option's own workers take them like local tasks, and so do the workers
// of CTAs that have found the option queue empty: such a CTA picks a board
// with posted work, rebuilds that option's tables from its Params, and works
// for it until the option ends.  Every task word carries the board's
// generation (bumped when the slot publishes an option and when the option
// ends) above its TASK_* state, so a claim for an option that has ended
// fails and a helper leaves as soon as the generation moves.
struct GTask {
    Buf in, out;
    int64_t x_lo, x_hi, g;
    int32_t lgN;
    volatile int32_t err;                 // status of the worker that ran it (0 = none)
    volatile unsigned long long posted_ns;   // when it was posted (global timer)
    unsigned long long word;              // gen << 2 | TASK_* state
};
struct Board {
    GTask t[kMaxDepth];
    volatile long long opt;               // option being priced (-1: none)
    volatile unsigned long long gen;
    volatile int tilt;                    // the option's convolutions are tilted
    unsigned mask;                        // bit d: t[d] posted and not yet claimed
    int helpers;                          // helping CTAs working for this option now
};
__device__ __forceinline__ unsigned long long gword(unsigned long long gen, int st) {
    return gen << 2 | (unsigned long long)st;
}


// Bound of the walker's and the workers' waits: AOP_FLAG_TEST_STALL (a test of
// the failure path: no worker takes a task) shortens it so that the first wait
// gives up quickly with AOP_ETIMEOUT.
__device__ __forceinline__ uint64_t wait_limit(const DncArgs &a) {
    return (a.flags & AOP_FLAG_TEST_STALL) ? kStallNs : kWaitNs;
}

// Serving: claim the next published request, or -1 when the host asks the
// kernel to stop or nothing is published for kIdleNs (the host relaunches the
// kernel on its next request).  A request is claimed only once published, so
// an exit never strands one.
constexpr uint64_t kIdleNs = 2000000000ull;
__device__ int64_t claim_published(const DncArgs &a) {
    const uint64_t t0 = gtime();
    for (;;) {
        const unsigned long long q = *(volatile unsigned long long *)a.sclaim;
        const long long p = *a.spub;
        if ((long long)q < p) {
            if (atomicCAS(a.sclaim, q, q + 1) == q) {
                __threadfence_system();      // the request's fields after its publication
                return (int64_t)q;
            }
            continue;
        }
        if (*a.sstop) return -1;
        if (gtime() - t0 > kIdleNs) return -1;
        __nanosleep(1000);
    }
}

struct Counters {
    long long convs, fft_points, fft_flops, conv_in, conv_out, base_cells, gbytes, wait_ns, busy_ns, base_ns;
    long long base_calls, base_rows, walker_ns, spec_ns, spec_bins, loop_cyc, fill_cyc;
    long long hist_n[24], hist_ns[24];   // linear advances by transform size log2 N
    long long cv_cyc[5];                 // single-tile advances: spectrum, stage, forward+product, inverse, store
    long long helped, helped_ns;         // advances run for another CTA's option
};

union TiltEntry {
    float2 f;
    double d;
};

// Per-CTA shared state (static shared memory).
struct Shared {
    ExpTables E;
    Params P;
    Task tasks[kMaxDepth];
    SpecEntry spec[kSpecSlots];
    int spec_n;
    int spec_lock;
    volatile unsigned posted;   // bit d: task slot d holds a posted task (idle workers scan this word)
    // direct index of the entries with g = Bodd * 2^k: entry + 1 (0 = none)
    volatile int16_t spec_map[kSpecLg][kSpecLg];
    long long arena_used;
    int opt;
    int helping;          // the option queue is empty: this CTA works for other options' boards
    int hk;               // board being helped (-1 none, -2 stop)
    int htilt;            // that option's tilt
    unsigned long long gen;   // generation of the option this CTA works for (own or helped)
    volatile int done;
    volatile int err;
    int bcast_i;
    long long bcast_l;
    double price;
    // e^{+-kappa n} = t2[n >> 14] t1[(n >> 7) & 127] t0[n & 127] in doubled
    // FP32 (FP32-split calls)
    // (FP64 in the FP64 mode, doubled FP32 otherwise: one 8-byte entry each)
    TiltEntry tup0[128], tup1[128], tup2[256];
    TiltEntry tdn0[128], tdn1[128], tdn2[256];
    int tilt_nmax;        // largest n with e^{kappa n} inside the entries' range
    // doubled-FP32 copies for the base cases of the FP32 modes: u^j, j < kNaiveCap
    float2 updf[kNaiveCap];
    float2 wdf[3];
    float2 kdf;
};

static_assert(kMaxDepth <= 32, "task slots are bits of Shared::posted");

// Tilt tables of the current option (all threads of the block).
template <int MODE>
__device__ void build_tilt_tables(Shared &S) {
    const double kap = S.P.kappa;
    for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
        const int dir = t >> 9, u = t & 511;
        const int lvl = u < 128 ? 0 : (u < 256 ? 1 : 2);
        const int j = lvl == 0 ? u : (lvl == 1 ? u - 128 : u - 256);
        const double e = kap * (double)j * (double)(1 << (7 * lvl));
        const double v = exp(dir ? -e : e);
        TiltEntry *tab = dir ? (lvl == 0 ? S.tdn0 : (lvl == 1 ? S.tdn1 : S.tdn2))
                             : (lvl == 0 ? S.tup0 : (lvl == 1 ? S.tup1 : S.tup2));
        if (MODE == 0) {
            tab[j].d = v;
        } else {
            const float h = (float)v;
            tab[j].f = isfinite(h) ? make_float2(h, (float)(v - (double)h)) : make_float2(h, 0.0f);
        }
    }
    const double range = (MODE == 0) ? 700.0 : 87.0;     // log of the largest factor kept
    if (threadIdx.x == 0) S.tilt_nmax = (int)fmin(range / kap, (double)((1 << 22) - 1));
}

// ---------------------------------------------------------------- groups
template <class G> __device__ __forceinline__ int bcast_int(Shared &S, int v);
template <> __device__ __forceinline__ int bcast_int<fft::WarpGroup>(Shared &, int v) {
    return __shfl_sync(0xffffffffu, v, 0);
}
template <> __device__ __forceinline__ int bcast_int<fft::BlockGroup>(Shared &S, int v) {
    if (threadIdx.x == 0) S.bcast_i = v;
    __syncthreads();
    int r = S.bcast_i;
    __syncthreads();
    return r;
}
template <class G> __device__ __forceinline__ bool leader() { return G::rank() == 0; }

// ------------------------------------------------------------ kernel power
__device__ int band_mc(const Params &P, int64_t g, int64_t N, bool tilt) {
    const double *w = tilt ? P.wt : P.w;
    const double wsum = tilt ? P.wtsum : P.wsum;
    const double w0 = w[0], w1 = w[1], w2 = w[2];
    double kap = 4.0 * (w0 * w1 + (P.nw == 3 ? w1 * w2 : 0.0)) / (wsum * wsum);
    double need = 83.2 / ((double)g * kap);
    if (!(kap > 0) || need >= 1.0) return (int)(N / 2);
    double th2 = asin(sqrt(need));               // theta_c / 2
    double mc = (double)N * th2 / 3.141592653589793 + 2.0;
    return (int)min((double)(N / 2), ceil(mc));
}

// s(theta_m)^g in FP64: magnitude through log1p of the exactly formed
// 1 - |s/s(0)|^2, phase g * arg s reduced in units of pi.
__device__ __noinline__ double2 bin_value(const Params &P, int64_t g, int lgN, int64_t m, bool tilt) {
    const double N = (double)((int64_t)1 << lgN);
    const double *w = tilt ? P.wt : P.w;
    const double wsum = tilt ? P.wtsum : P.wsum;
    const double w0 = w[0], w1 = w[1], w2 = w[2];
    const double inv2 = 1.0 / (wsum * wsum);
    const double gd = (double)g;
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
    // 1 - |s/s(0)|^2 lies in [0, 1]; rounding can step outside when |s(pi)|
    // vanishes (e.g. p = 1/2), where the power is zero anyway
    dl = fmin(fmax(dl, 0.0), 1.0);
    double lm = (dl >= 1.0) ? -INFINITY : gd * (log(wsum) + 0.5 * log1p(-dl));
    double ph = gd * atan2(im, re);
    double phpi = ph * 0.3183098861837907;
    phpi -= 2.0 * rint(0.5 * phpi);
    double sp, cp;
    sincospi(phpi, &sp, &cp);
    double mag = (lm < -745.0) ? 0.0 : exp(lm);
    return make_double2(mag * cp, mag * sp);
}

template <int MODE>
__device__ __forceinline__ typename fft::Cx<MODE>::Sp pack_spec(double2 v) {
    if constexpr (MODE == 0) {
        return v;
    } else {
        float hr = (float)v.x, hi = (float)v.y;
        return make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
    }
}

// ------------------------------------------------------- storage policies
// How a linear advance reads its input and writes its output:
//   StoreF64  -- plain FP64 arrays (the linear-advance entry points);
//   StoreCell -- the pricer's row buffers (FP64 in mode 0, FP32 pairs else),
//                read and written without FP64 arithmetic in modes 1 and 2.
template <int MODE>
struct StoreF64 {
    using T = double;
    using V = typename fft::Cx<MODE>::V;
    static constexpr bool kIdentity = false;
    __device__ static V to_v(double d) { return fft::load_split<MODE>(d); }
    __device__ static double from_v(V v, const ConvScale &cs) { return fft::unsplit(v, cs.d); }
};
template <int MODE>
struct StoreCell {
    using T = typename fft::CellT<MODE>::T;
    using V = typename fft::Cx<MODE>::V;
    static constexpr bool kIdentity = (MODE == 1);
    __device__ static V to_v(T c) {
        if constexpr (MODE == 0) return fft::cell_to_v(c);
        else if constexpr (MODE == 1) return fft::cell_to_v1(c);
        else return fft::cell_to_v2(c);
    }
    __device__ static T from_v(V v, const ConvScale &cs) { return fft::v_to_cell(v, cs.d, cs.f); }
};

// ------------------------------------------------------------- per-CTA view
template <int MODE>
struct Cta {
    using V = typename fft::Cx<MODE>::V;
    using Tw = typename fft::Cx<MODE>::Tw;
    using Sp = typename fft::Cx<MODE>::Sp;

    const DncArgs &a;
    Shared &S;
    char *slot;
    bool tilt = false;    // exponential tilt of the call convolutions
    long long cnt_spec_ns = 0, cnt_spec_bins = 0;   // spectrum builds by this thread's group

    __device__ Cta(const DncArgs &a_, Shared &S_, char *slot_) : a(a_), S(S_), slot(slot_) {}
    // base-case height of the current option
    __device__ int bcase() const { return S.P.model == AOP_BSM_PUT ? a.Bput : a.B; }

    // e^{+kappa n} (0 past the float range) and e^{-kappa n} from the
    // tables, in doubled FP32
    __device__ static float2 df_prod(float2 a, float2 b) {
        float h, l;
        fft::df_mul(a.x, a.y, b.x, b.y, h, l);
        return make_float2(h, l);
    }
    __device__ float2 tilt_up(int64_t n) const {
        if (n > S.tilt_nmax) return make_float2(0.0f, 0.0f);
        return df_prod(df_prod(S.tup2[n >> 14].f, S.tup1[(n >> 7) & 127].f), S.tup0[n & 127].f);
    }
    __device__ double tilt_up64(int64_t n) const {
        if (n > S.tilt_nmax) return 0.0;
        return S.tup2[n >> 14].d * S.tup1[(n >> 7) & 127].d * S.tup0[n & 127].d;
    }
    __device__ double tilt_dn64(int64_t n) const {
        if ((n >> 14) > 255) return 0.0;
        return S.tdn2[n >> 14].d * S.tdn1[(n >> 7) & 127].d * S.tdn0[n & 127].d;
    }
    __device__ float2 tilt_dn(int64_t n) const {
        if ((n >> 14) > 255) return make_float2(0.0f, 0.0f);
        return df_prod(df_prod(S.tdn2[n >> 14].f, S.tdn1[(n >> 7) & 127].f), S.tdn0[n & 127].f);
    }
    // output cell y = x_hi - n of a tilted advance: multiply by e^{-kappa n}
    template <class ST>
    __device__ typename ST::T untilt(typename ST::T c, int64_t n, const ConvScale &cs) const {
        if (!tilt) return c;
        const int64_t m = max(n - cs.n0, (int64_t)0);
        if constexpr (MODE == 0) {
            return c * (tilt_dn64(m) * cs.resid64);
        } else if constexpr (std::is_same<typename ST::T, float2>::value) {
            const float2 f = df_prod(tilt_dn(m), cs.resid);
            float h, l;
            fft::two_sum(c.x, c.y, h, l);
            return df_prod(make_float2(h, l), f);
        } else {
            return c;
        }
    }
    // a staged input value of column x = x_hi - n times e^{+kappa n}
    __device__ V tilt_in(V v, int64_t n) const {
        if constexpr (MODE == 0) {
            v.x *= tilt_up64(n);
            return v;
        } else if constexpr (MODE == 1) {
            const float2 f = tilt_up(n);
            float h, l;
            fft::two_sum(v.x, v.y, h, l);
            return df_prod(make_float2(h, l), f);
        } else {
            const float2 f = tilt_up(n);
            float h, l;
            fft::two_sum(v.v.x, v.v.z, h, l);
            const float2 p = df_prod(make_float2(h, l), f);
            v.v.x = p.x;
            v.v.z = p.y;
            return v;
        }
    }

    __device__ const Params &P() const { return S.P; }
    __device__ double *mid(int d) const { return (double *)(slot + a.off_mid) + a.mid_off[d]; }
    __device__ V *scratch(int w) const { return (V *)(slot + a.off_scr + (int64_t)w * a.scr_stride); }
    __device__ Sp *arena() const { return (Sp *)(slot + a.off_spec); }
    __device__ const Tw *tw() const { return (const Tw *)a.tw; }
    __device__ Board *board_of(int64_t k) const { return (Board *)(a.ws + k * a.ws_stride + a.off_board); }
    __device__ Board *board() const { return (Board *)(slot + a.off_board); }
    // board threshold (0: no helping); compiled out of the FP32-split mode,
    // whose 128-register budget the board code would spill into
    __device__ int help_lg() const { return MODE == 1 ? 0 : a.help_lg; }

    // Cached kernel power for (g, lgN); nullptr = evaluate bins on the fly
    // (arena exhausted).  Called by every thread of the group G.
    template <class G>
    __device__ const Sp *spectrum(int64_t g, int lgN, int &mc_out, ConvScale &cs) {
        // fast path: a ready entry found through the direct index, no lock.
        // The recursion's heights are the base-case height times powers of
        // two, so g = Bodd * 2^lgg with Bodd the odd part of B.
        const int lgg = g > 0 ? __ffsll((long long)g) - 1 : 0;
        const int bc = bcase();
        const bool direct = g > 0 && bc > 0 && (g >> lgg) == (bc >> (__ffs(bc) - 1)) && lgN < kSpecLg &&
                            lgg < kSpecLg;
        if (direct) {
            const int v = S.spec_map[lgg][lgN];
            if (v > 0) {
                SpecEntry &e = S.spec[v - 1];
                if (e.state == SPEC_READY) {
                    __threadfence_block();
                    mc_out = e.mc;
                    cs.n0 = e.n0;
                    cs.resid = e.resid;
                    cs.resid64 = e.resid64;
                    return arena() + e.off;
                }
            }
        }
        int idx = -1, build = 0;
        if (leader<G>()) {
            const uint64_t t0 = gtime();
            while (atomicCAS(&S.spec_lock, 0, 1) != 0) {
                __nanosleep(32);
                if (gtime() - t0 > kWaitNs) { atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT); break; }
            }
            for (int i = 0; i < S.spec_n; i++)
                if (S.spec[i].g == (int32_t)g && S.spec[i].lgN == lgN) { idx = i; break; }
            if (idx < 0) {
                int mc = band_mc(P(), g, (int64_t)1 << lgN, tilt);
                if (S.spec_n < kSpecSlots && S.arena_used + mc + 1 <= a.spec_cap) {
                    idx = S.spec_n;
                    S.spec[idx].g = (int32_t)g;
                    S.spec[idx].lgN = lgN;
                    S.spec[idx].mc = mc;
                    S.spec[idx].off = S.arena_used;
                    S.spec[idx].n0 = 0;
                    S.spec[idx].resid = make_float2(1.0f, 0.0f);
                    S.spec[idx].resid64 = 1.0;
                    if (tilt) tilt_shift(P(), g, S.spec[idx].n0, S.spec[idx].resid, S.spec[idx].resid64);
                    S.spec[idx].state = SPEC_BUILDING;
                    S.arena_used += mc + 1;
                    __threadfence_block();
                    S.spec_n = idx + 1;
                    if (direct) S.spec_map[lgg][lgN] = (int16_t)(idx + 1);
                    build = 1;
                } else {
                    idx = -1 - mc;   // no room: evaluate on the fly
                }
            }
            __threadfence_block();
            atomicExch(&S.spec_lock, 0);
        }
        idx = bcast_int<G>(S, idx);
        build = bcast_int<G>(S, build);
        if (idx < 0) {
            mc_out = -1 - idx;
            cs.n0 = 0;
            cs.resid = make_float2(1.0f, 0.0f);
            cs.resid64 = 1.0;
            if (tilt) tilt_shift(P(), g, cs.n0, cs.resid, cs.resid64);
            return nullptr;
        }
        SpecEntry &e = S.spec[idx];
        Sp *p = arena() + e.off;
        if (build) {
            const uint64_t ts0 = gtime();
            for (int m = G::rank(); m <= e.mc; m += G::size()) p[m] = pack_spec<MODE>(bin_value(P(), g, lgN, m, tilt));
            __threadfence_block();
            G::sync();
            if (leader<G>()) {
                e.state = SPEC_READY;
                cnt_spec_ns += (long long)(gtime() - ts0);
                cnt_spec_bins += e.mc + 1;
            }
        } else if (leader<G>()) {
            const uint64_t t0 = gtime();
            while (e.state != SPEC_READY) {
                __nanosleep(32);
                if (gtime() - t0 > kWaitNs) { atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT); break; }
            }
            __threadfence_block();
        }
        G::sync();
        mc_out = e.mc;
        cs.n0 = e.n0;
        cs.resid = e.resid;
        cs.resid64 = e.resid64;
        return p;
    }

    // Fill tile[s] (s < count) with the stored input value at transform index
    // e = idx(s) (zero past the window W), converted by the storage policy ST
    // (8-byte stored values).  The values are staged with cp.async (all in
    // flight at once; padding is zero-filled, not read) and converted in shared
    // memory: in place for 8-byte transform values; 16-byte values are staged
    // in the upper half of the tile and converted in rounds of 16 values a
    // thread, each round read into registers before any of it is written (a
    // round's writes only cover staged values of that round or earlier ones).
    template <class G, class ST, class IDX>
    __device__ void stage_input(V *tile, int count, IDX idx, const Buf &in, int64_t x_lo, int64_t W) {
        using T = typename ST::T;
        static_assert(sizeof(T) == 8, "stored values are 8 bytes");
        const T *src = (const T *)in.p - in.base;
        if constexpr (sizeof(V) == 8) {
            for (int s = G::rank(); s < count; s += G::size()) {
                const int e = idx(s);
                const bool ok = e < W;
                fft::cp_async<8>(&tile[s], ok ? (const void *)&src[x_lo + e] : (const void *)in.p, ok ? 8 : 0);
            }
            fft::cp_async_wait();
            if constexpr (!ST::kIdentity) {
                for (int s = G::rank(); s < count; s += G::size()) {
                    const T d = *(const T *)&tile[s];
                    tile[s] = ST::to_v(d);
                }
            }
            if (tilt) {
                for (int s = G::rank(); s < count; s += G::size()) {
                    const int e = idx(s);
                    if (e < W) tile[s] = tilt_in(tile[s], W - 1 - e);
                }
            }
        } else {
            constexpr int kPer = 16;
            T *st = (T *)tile + count;
            for (int s = G::rank(); s < count; s += G::size()) {
                const int e = idx(s);
                const bool ok = e < W;
                fft::cp_async<8>(&st[s], ok ? (const void *)&src[x_lo + e] : (const void *)in.p, ok ? 8 : 0);
            }
            fft::cp_async_wait();
            for (int base = 0; base < count; base += kPer * G::size()) {
                T r[kPer];
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    const int s = base + G::rank() + k * G::size();
                    if (s < count) r[k] = st[s];
                }
                G::sync();
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    const int s = base + G::rank() + k * G::size();
                    if (s < count) {
                        tile[s] = ST::to_v(r[k]);
                        if (tilt) {
                            const int e = idx(s);
                            if (e < W) tile[s] = tilt_in(tile[s], W - 1 - e);
                        }
                    }
                }
                G::sync();
            }
        }
        G::sync();
    }

    template <class ST>
    __device__ static void store(const Buf &out, int64_t y, typename ST::T v) {
        ((typename ST::T *)out.p)[y - out.base] = v;
    }

    // tile[s] = scr[idx(s)] for s < count, through cp.async
    template <class G, class IDX>
    __device__ void stage_scratch(V *tile, int count, IDX idx, const V *scr) {
        for (int s = G::rank(); s < count; s += G::size())
            fft::cp_async<(int)sizeof(V)>(&tile[s], &scr[idx(s)], (int)sizeof(V));
        fft::cp_async_wait();
        G::sync();
    }

    // tile[s] times the kernel power of bin brev(base + s), s < count, for the
    // group G.  Each thread loads the spectrum entries of four of its bins
    // before it multiplies any, so that their global-memory latencies overlap
    // (one at a time, they serialised the product).  Out of line: one copy for
    // the single-tile and the multi-pass transforms.
    template <class G>
    __device__ __noinline__ void product(V *tile, int count, uint32_t base, int lgN, const Sp *sp, int mc,
                                         int64_t g) {
        const uint32_t N = 1u << lgN;
        if (!sp) {
            for (int s = G::rank(); s < count; s += G::size())
                tile[s] = mul_bin(tile[s], sp, mc, fft::brev_n(base + (uint32_t)s, lgN), N, g, lgN);
            G::sync();
            return;
        }
        constexpr int kB = 4;
        for (int s0 = G::rank(); s0 < count; s0 += kB * G::size()) {
            Sp w[kB];
            uint32_t m[kB];
#pragma unroll
            for (int j = 0; j < kB; j++) {
                const int s = s0 + j * G::size();
                m[j] = fft::brev_n(base + (uint32_t)s, lgN);
                const uint32_t mm = (m[j] <= N / 2) ? m[j] : N - m[j];
                if (s < count && (int)mm <= mc) w[j] = sp[mm];   // written by this CTA: plain (coherent) load
                else m[j] = 0xffffffffu;            // outside the band: zero
            }
#pragma unroll
            for (int j = 0; j < kB; j++) {
                const int s = s0 + j * G::size();
                if (s >= count) break;
                if (m[j] == 0xffffffffu) tile[s] = fft::czero<V>();
                else tile[s] = (m[j] <= N / 2) ? fft::twmul<false>(tile[s], w[j]) : fft::twmul<true>(tile[s], w[j]);
            }
        }
        G::sync();
    }

    // Real-input form of a single-tile advance (16-byte transform values, whose
    // imaginary half would otherwise carry zeros): the N real cells are staged
    // as M = N/2 complex values z[s] = x[2s] + i x[2s+1]; after the M-point
    // forward transform Z, each pair of bins (k, M-k) gives the N-point
    // spectrum of the row, X[k] = E + W^k O and X[k+M] = E - W^k O with
    // E = (Z[k] + conj Z[M-k])/2, O = (Z[k] - conj Z[M-k])/(2i), W = e^{-2 pi i/N};
    // times the kernel power Y = X S, it is folded back into
    // Z''[k] = (Y[k] + Y[k+M]) + i W^{-k} (Y[k] - Y[k+M]), whose M-point inverse
    // is N (y[2s] + i y[2s+1]) (Y is Hermitian, so the pair's second bin is
    // Z''[M-k] = conj(A) + i W^k conj(B) with A, B the sum and difference).
    // Stage the cells 2e and 2e + 1 (e = idx(s)) of the window as tile[s] =
    // x[2e] + i x[2e+1] (zero past W).  The two 8-byte cells land in the bytes
    // of tile[s] and are converted in place by the thread that loaded them.
    template <class G, class ST, class IDX>
    __device__ void stage_packed(V *tile, int count, IDX idx, const Buf &in, int64_t x_lo, int64_t W) {
        using C = typename ST::T;                      // an 8-byte stored cell
        static_assert(sizeof(C) == 8, "stored values are 8 bytes");
        const C *src = (const C *)in.p - in.base;
        for (int s = G::rank(); s < count; s += G::size()) {
            const int64_t c = 2 * (int64_t)idx(s);
            const bool ok0 = c < W, ok1 = c + 1 < W;
            fft::cp_async<8>((C *)tile + 2 * s, ok0 ? (const void *)&src[x_lo + c] : (const void *)in.p, ok0 ? 8 : 0);
            fft::cp_async<8>((C *)tile + 2 * s + 1, ok1 ? (const void *)&src[x_lo + c + 1] : (const void *)in.p,
                             ok1 ? 8 : 0);
        }
        fft::cp_async_wait();
        for (int s = G::rank(); s < count; s += G::size()) {
            const int64_t c = 2 * (int64_t)idx(s);
            const C c0 = ((const C *)tile)[2 * s], c1 = ((const C *)tile)[2 * s + 1];
            V v0 = ST::to_v(c0), v1 = ST::to_v(c1);
            if (tilt) {
                if (c < W) v0 = tilt_in(v0, W - 1 - c);
                if (c + 1 < W) v1 = tilt_in(v1, W - 2 - c);
            }
            if constexpr (MODE == 0) {
                tile[s] = make_double2(v0.x, v1.x);
            } else {
                fft::df2 r;
                r.v = make_float4(v0.v.x, v1.v.x, v0.v.z, v1.v.z);
                tile[s] = r;
            }
        }
        G::sync();
    }
    // Output cell c (= 2e or 2e + 1) of element value v of a real transform
    __device__ static V packed_part(V v, int64_t c) {
        if (c & 1) {
            if constexpr (MODE == 0) v = make_double2(v.y, 0.0);
            else v.v = make_float4(v.v.y, 0.f, v.v.w, 0.f);
        }
        return v;
    }
    // The split-product-merge step on blocks of 2^lti bins of an M-point
    // transform (M = 2^lgM) stored in bit-reversed order: the block of residue
    // rb holds bins k = rb + (brev(s) << (lgM - lti)); bin M - k lies in the
    // mirror block at slot s ^ (2^lti - 1) (held at tile + 2^lti when `two`),
    // or, for the blocks of residue 0 and 2^(lgM-lti-1), in the same block.
    template <class G>
    __device__ void real_pairs(V *tile, bool two, int rb, int lgM, int lti, const Sp *sp, int mc, int64_t g) {
        const uint32_t M = 1u << lgM, N = 2u * M;
        const int lgN = lgM + 1;
        const int Bs = 1 << lti, mask = Bs - 1, nbl = lgM - lti;
        const Tw *T = tw();
        auto pair = [&](int pk, int pj, uint32_t k) {
            const V zk = tile[pk], cj = fft::cconj(tile[pj]);
            const V E = fft::chalf(fft::cadd(zk, cj));
            const V O = fft::chalf(fft::cmul_mi(fft::csub(zk, cj)));
            const Tw w = fft::tw_get<MODE>(T, a.tw_log2, k, lgN);     // W^k, k < M
            const V wo = fft::twmul<false>(O, w);
            const V yk = mul_bin(fft::cadd(E, wo), sp, mc, k, N, g, lgN);
            const V ym = mul_bin(fft::csub(E, wo), sp, mc, k + M, N, g, lgN);
            const V A = fft::cadd(yk, ym), B = fft::csub(yk, ym);
            tile[pk] = fft::cadd(A, fft::cmul_pi(fft::twmul<true>(B, w)));
            if (pj != pk) tile[pj] = fft::cadd(fft::cconj(A), fft::cmul_pi(fft::twmul<false>(fft::cconj(B), w)));
        };
        if (two) {
            for (int s = G::rank(); s < Bs; s += G::size())
                pair(s, Bs + (s ^ mask), (uint32_t)rb + (fft::brev_n((uint32_t)s, lti) << nbl));
        } else if (rb == 0) {
            for (int kp = G::rank(); kp <= Bs / 2; kp += G::size())
                pair((int)fft::brev_n((uint32_t)kp, lti), (int)fft::brev_n((uint32_t)((Bs - kp) & mask), lti),
                     (uint32_t)kp << nbl);
        } else {
            for (int s = G::rank(); s < Bs / 2; s += G::size())
                pair(s, s ^ mask, (uint32_t)rb + (fft::brev_n((uint32_t)s, lti) << nbl));
        }
        G::sync();
    }

    __device__ V mul_bin(V z, const Sp *sp, int mc, uint32_t m, uint32_t N, int64_t g, int lgN) const {
        if (sp) return fft::spec_mul<MODE>(z, sp, mc, m, N);
        uint32_t mm = (m <= N / 2) ? m : N - m;
        if ((int)mm > mc) return fft::czero<V>();
        Sp s = pack_spec<MODE>(bin_value(P(), g, lgN, mm, tilt));
        return (m <= N / 2) ? fft::twmul<false>(z, s) : fft::twmul<true>(z, s);
    }

    // One pass over global memory: the stages with half-sizes 2^s_lo .. 2^s_hi
    // of an N-point transform, on tiles of (2^(s_hi-s_lo+1) elements x Q
    // consecutive columns) staged in shared memory, radix-4 inside the tile.
    // DIF = forward (stages top down); otherwise inverse.  The first forward
    // pass reads (and splits) the FP64 input; the last inverse pass extracts
    // the FP64 output.
    template <class G, class ST, bool DIF, bool REAL = false>
    __device__ void tile_pass(V *tile, int lg_tile, V *scr, int lgN, int s_lo, int s_hi, bool first, bool last,
                              const Buf &in, int64_t x_lo, int64_t W, const Buf &out, int64_t y_lo, int64_t off,
                              int64_t nout, const ConvScale &cs) {
        const int L = s_hi - s_lo + 1;
        const int lgQ = min(s_lo, lg_tile - L);
        const int qm = (1 << lgQ) - 1;
        const int count = 1 << (L + lgQ);
        const int lo_count = 1 << s_lo;
        const int hi_count = 1 << (lgN - s_hi - 1);
        const Tw *T = tw();
        for (int hb = 0; hb < hi_count; hb++) {
            const int hbase = hb << (s_hi + 1);
            for (int q0 = 0; q0 < lo_count; q0 += qm + 1) {
                auto idx = [=](int s) { return hbase + ((s >> lgQ) << s_lo) + q0 + (s & qm); };
                if (first) {
                    if constexpr (REAL) stage_packed<G, ST>(tile, count, idx, in, x_lo, W);
                    else stage_input<G, ST>(tile, count, idx, in, x_lo, W);
                } else {
                    stage_scratch<G>(tile, count, idx, scr);
                }
                const fft::Cols cl{lgQ, s_lo, q0};
                if (a.radix2) {
                    if (DIF) fft::dif_cols_r2<MODE, G>(tile, L, L - 1, 0, cl, T);
                    else fft::dit_cols_r2<MODE, G>(tile, L, 0, L - 1, cl, T);
                } else {
                    if (DIF) fft::dif_cols<MODE, G>(tile, L, L - 1, 0, cl, T);
                    else fft::dit_cols<MODE, G>(tile, L, 0, L - 1, cl, T);
                }
                for (int s = G::rank(); s < count; s += G::size()) {
                    const int e = idx(s);
                    if (last) {
                        if constexpr (REAL) {
                            for (int h = 0; h < 2; h++) {      // cells 2e and 2e + 1
                                const int64_t k = 2 * (int64_t)e + h - off;
                                if (k >= 0 && k < nout)
                                    store<ST>(out, y_lo + k,
                                              untilt<ST>(ST::from_v(packed_part(tile[s], h), cs), W - 1 - k, cs));
                            }
                        } else {
                            const int64_t k = e - off;
                            if (k >= 0 && k < nout)
                                store<ST>(out, y_lo + k, untilt<ST>(ST::from_v(tile[s], cs), W - 1 - k, cs));
                        }
                    } else {
                        scr[e] = tile[s];
                    }
                }
                G::sync();
            }
        }
    }

    // Linear advance of `g` steps: out[y] = sum_t c_t in[y + o_min g + t] for y
    // in [x_lo - o_min g, x_hi - (o_min + nw - 1) g].  The group G runs it on its
    // shared tile (2^lg_tile values) and, for longer transforms, on its global
    // scratch `scr`.
    // returns log2 of the transform length (0: nothing to do)
    template <class G, class ST>
    __device__ int conv(const Buf &in, int64_t x_lo, int64_t x_hi, const Buf &out, int64_t g, V *tile,
                        int lg_tile, V *scr, Counters &cnt) {
        const Params &Pp = P();
        const int64_t W = x_hi - x_lo + 1;
        const int64_t span = (int64_t)(Pp.nw - 1) * g;
        const int64_t y_lo = x_lo - (int64_t)Pp.o_min * g;
        const int64_t nout = W - span;
        if (nout <= 0) return 0;
        int lgN = ilog2_ceil(W);
        if (lgN < 2) lgN = 2;
        const int64_t N = (int64_t)1 << lgN;
        int mc;
        ConvScale cs;
        const long long q0 = clock64();
        const Sp *sp = spectrum<G>(g, lgN, mc, cs);
        cs.d = __longlong_as_double((long long)(1023 - lgN) << 52);
        cs.f = __int_as_float((127 - lgN) << 23);
        const int64_t off = y_lo - x_lo;
        if (leader<G>()) {
            cnt.convs++;
            cnt.fft_points += 2 * N;
            cnt.fft_flops += 2 * 5 * N * lgN;
            cnt.conv_in += W;
            cnt.conv_out += nout;
        }
        const Tw *T = tw();
        if constexpr (sizeof(V) == 16) {
            if (lgN <= lg_tile + 1) {                     // N/2 complex points fit the tile
                const long long q1 = clock64();
                stage_packed<G, ST>(tile, (int)N / 2, [](int s) { return s; }, in, x_lo, W);
                const long long q2 = clock64();
                fft::dif_all<MODE, G>(tile, lgN - 1, T, a.radix2);
                real_pairs<G>(tile, false, 0, lgN - 1, lgN - 1, sp, mc, g);
                const long long q3 = clock64();
                fft::dit_all<MODE, G>(tile, lgN - 1, T, a.radix2);
                const long long q4 = clock64();
                for (int64_t t = G::rank(); t < nout; t += G::size()) {
                    const int64_t p = off + t;            // odd cells in the imaginary part
                    store<ST>(out, y_lo + t, untilt<ST>(ST::from_v(packed_part(tile[p >> 1], p), cs), W - 1 - t, cs));
                }
                G::sync();
                if (leader<G>()) {
                    const long long q5 = clock64();
                    cnt.cv_cyc[0] += q1 - q0;
                    cnt.cv_cyc[1] += q2 - q1;
                    cnt.cv_cyc[2] += q3 - q2;
                    cnt.cv_cyc[3] += q4 - q3;
                    cnt.cv_cyc[4] += q5 - q4;
                }
                return lgN;
            }
        }
        if (lgN <= lg_tile) {
            const long long q1 = clock64();
            stage_input<G, ST>(tile, (int)N, [](int s) { return s; }, in, x_lo, W);
            const long long q2 = clock64();
            fft::dif_all<MODE, G>(tile, lgN, T, a.radix2);
            product<G>(tile, (int)N, 0u, lgN, sp, mc, g);
            const long long q3 = clock64();
            fft::dit_all<MODE, G>(tile, lgN, T, a.radix2);
            const long long q4 = clock64();
            for (int64_t t = G::rank(); t < nout; t += G::size())
                store<ST>(out, y_lo + t, untilt<ST>(ST::from_v(tile[off + t], cs), W - 1 - t, cs));
            G::sync();
            if (leader<G>()) {
                const long long q5 = clock64();
                cnt.cv_cyc[0] += q1 - q0;
                cnt.cv_cyc[1] += q2 - q1;
                cnt.cv_cyc[2] += q3 - q2;
                cnt.cv_cyc[3] += q4 - q3;
                cnt.cv_cyc[4] += q5 - q4;
            }
            return lgN;
        }
        if constexpr (sizeof(V) == 16) {
            // the real row as an M = N/2-point complex transform: outer stages
            // lti .. lgM-1 over global memory, then the inner stages on pairs of
            // mirror blocks of 2^lti bins (half a tile each) around the
            // split-product-merge step
            const int lgM = lgN - 1, lti = lg_tile - 1;
            if (leader<G>()) cnt.gbytes += (int64_t)sizeof(V) * (N / 2) * 4 + 8 * (W + nout);
            const int chunk = max(1, lg_tile - 1);
            const int outer = lgM - lti;
            const int nch = min(16, (outer + chunk - 1) / chunk);
            int ch_lo[16], ch_hi[16];
            for (int c = 0, s_hi = lgM - 1; c < nch; c++) {
                const int len = outer / nch + (c < outer % nch ? 1 : 0);
                ch_hi[c] = s_hi;
                ch_lo[c] = s_hi - len + 1;
                s_hi -= len;
            }
            for (int c = 0; c < nch; c++)
                tile_pass<G, ST, true, true>(tile, lg_tile, scr, lgM, ch_lo[c], ch_hi[c], c == 0, false, in, x_lo, W,
                                             out, y_lo, off, nout, cs);
            const int Bs = 1 << lti, lgb = lgM - lti, nb = 1 << lgb;
            for (int b = 0; b < nb; b++) {
                const int rb = (int)fft::brev_n((uint32_t)b, lgb);
                const int b2 = (int)fft::brev_n((uint32_t)((nb - rb) & (nb - 1)), lgb);
                if (b2 < b) continue;                      // each mirror pair once
                const bool two = b2 != b;
                V *blk1 = scr + (int64_t)b * Bs, *blk2 = scr + (int64_t)b2 * Bs;
                const int cnt2 = two ? 2 * Bs : Bs;
                for (int s = G::rank(); s < cnt2; s += G::size())
                    fft::cp_async<(int)sizeof(V)>(&tile[s], s < Bs ? &blk1[s] : &blk2[s - Bs], (int)sizeof(V));
                fft::cp_async_wait();
                G::sync();
                fft::dif_all<MODE, G>(tile, lti, T, a.radix2);
                if (two) fft::dif_all<MODE, G>(tile + Bs, lti, T, a.radix2);
                real_pairs<G>(tile, two, rb, lgM, lti, sp, mc, g);
                fft::dit_all<MODE, G>(tile, lti, T, a.radix2);
                if (two) fft::dit_all<MODE, G>(tile + Bs, lti, T, a.radix2);
                for (int s = G::rank(); s < cnt2; s += G::size()) {
                    if (s < Bs) blk1[s] = tile[s];
                    else blk2[s - Bs] = tile[s];
                }
                G::sync();
            }
            for (int c = nch - 1; c >= 0; c--)
                tile_pass<G, ST, false, true>(tile, lg_tile, scr, lgM, ch_lo[c], ch_hi[c], false, c == 0, in, x_lo, W,
                                              out, y_lo, off, nout, cs);
            return lgN;
        }
        if (leader<G>()) cnt.gbytes += (int64_t)sizeof(V) * N * 4 + 8 * (W + nout);
        // outer stages lg_tile .. lgN-1 in as few passes as the tile allows,
        // balanced: a pass of L stages moves rows of Q = 2^(lg_tile - L)
        // consecutive values, at least 32 bytes (one DRAM sector)
        const int chunk = max(1, lg_tile - (sizeof(V) >= 16 ? 1 : 2));
        const int outer = lgN - lg_tile;
        const int nch = min(16, (outer + chunk - 1) / chunk);
        int ch_lo[16], ch_hi[16];
        for (int c = 0, s_hi = lgN - 1; c < nch; c++) {
            const int len = outer / nch + (c < outer % nch ? 1 : 0);
            ch_hi[c] = s_hi;
            ch_lo[c] = s_hi - len + 1;
            s_hi -= len;
        }
        for (int c = 0; c < nch; c++)
            tile_pass<G, ST, true>(tile, lg_tile, scr, lgN, ch_lo[c], ch_hi[c], c == 0, false, in, x_lo, W, out, y_lo,
                                   off, nout, cs);
        // inner stages on contiguous blocks, with the kernel-power product
        const int N2 = 1 << lg_tile;
        for (int b = 0; b < (int)(N / N2); b++) {
            V *blk = scr + (int64_t)b * N2;
            stage_scratch<G>(tile, N2, [](int s) { return s; }, blk);
            fft::dif_all<MODE, G>(tile, lg_tile, T, a.radix2);
            product<G>(tile, N2, (uint32_t)(b * N2), lgN, sp, mc, g);
            fft::dit_all<MODE, G>(tile, lg_tile, T, a.radix2);
            for (int s = G::rank(); s < N2; s += G::size()) blk[s] = tile[s];
            G::sync();
        }
        for (int c = nch - 1; c >= 0; c--)
            tile_pass<G, ST, false>(tile, lg_tile, scr, lgN, ch_lo[c], ch_hi[c], false, c == 0, in, x_lo, W, out, y_lo,
                                    off, nout, cs);
        return lgN;
    }
};

// ------------------------------------------------- base-case arithmetic
// The base cases step rows of up to kRegCells cells, one warp, D+1-point
// stencil with non-negative weights and values.  FP64 on this GPU issues one
// warp instruction per 64 cycles per SM sub-partition whatever the number of
// active lanes, so the FP32 modes step their base cases in doubled FP32
// (hi + lo, about 48 significant bits) on the FP32 pipe; the FP64 mode keeps
// FP64.
struct ArithF64 {
    using T = double;
    struct Wts { double w0, w1, w2; };
    __device__ static T zero() { return 0.0; }
    __device__ static Wts weights(const Shared &S) { return Wts{S.P.w[0], S.P.w[1], S.P.w[2]}; }
    template <int MODE> __device__ static T load(const Buf &b, int64_t x) { return cell_ld<MODE>(b, x); }
    template <int MODE> __device__ static void store(const Buf &b, int64_t x, T v) { cell_st<MODE>(b, x, v); }
    __device__ static T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    __device__ static T dot2(const Wts &w, T a, T b) { return w.w0 * a + w.w1 * b; }
    __device__ static T dot3(const Wts &w, T a, T b, T c) { return w.w0 * a + w.w1 * b + w.w2 * c; }
    // continuation >= exercise for a non-negative continuation, decided on the
    // bit patterns (non-negative doubles order like their integer images)
    __device__ static bool cont_ge(T cont, T ex) {
        const long long eb = __double_as_longlong(ex);
        return eb <= 0 || __double_as_longlong(cont) >= eb;
    }
    // exercise > continuation > = 0 (put), on the bit patterns likewise
    __device__ static bool ex_gt(T ex, T cont) {
        const long long eb = __double_as_longlong(ex);
        return eb > 0 && eb > __double_as_longlong(cont);
    }
    // exercise values of exponent indices klo .. khi into ext (one warp)
    __device__ static void fill(const Shared &S, T *ext, int64_t klo, int64_t khi, int lane) {
#pragma unroll 4
        for (int64_t kp = klo + lane; kp <= khi; kp += 32) ext[kp - klo] = aop::exercise(S.P, S.E, kp);
    }
};

struct ArithDF {
    using T = float2;      // hi + lo, normalised (|lo| <= ulp(hi) / 2)
    struct Wts { float2 w0, w1, w2; };
    __device__ static T zero() { return make_float2(0.f, 0.f); }
    __device__ static Wts weights(const Shared &S) { return Wts{S.wdf[0], S.wdf[1], S.wdf[2]}; }
    // a stored cell (FP32 pair, from a base case or an FFT advance) renormalised
    template <int MODE> __device__ static T load(const Buf &b, int64_t x) {
        const float2 c = ((const float2 *)b.p)[x - b.base];
        float s, e;
        fft::two_sum(c.x, c.y, s, e);
        return make_float2(s, e);
    }
    template <int MODE> __device__ static void store(const Buf &b, int64_t x, T v) {
        ((float2 *)b.p)[x - b.base] = v;
    }
    __device__ static T shfl(T v, int src) {
        return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
    }
    // fused dot products of the stencil (fft.cuh)
    __device__ static T dot2(const Wts &w, T a, T b) { return fft::df_dot2(w.w0, w.w1, a, b); }
    __device__ static T dot3(const Wts &w, T a, T b, T c) { return fft::df_dot3(w.w0, w.w1, w.w2, a, b, c); }
    __device__ static bool ge(T a, T b) { return fft::df_ge(a, b); }
    __device__ static bool pos(T a) { return a.x > 0.f || (a.x == 0.f && a.y > 0.f); }
    __device__ static bool cont_ge(T cont, T ex) { return !pos(ex) || ge(cont, ex); }
    __device__ static bool ex_gt(T ex, T cont) { return pos(ex) && !ge(cont, ex); }
    // exercise values S u^k - K (calls) or 1 - e^{s_k} (put) of exponent
    // indices klo .. khi: the node price at klo once in FP64, then
    // e^{x_klo} u^j from the doubled-FP32 table (khi - klo < kNaiveCap, and
    // the caller keeps u^(khi - klo) inside the float range)
    __device__ static void fill(const Shared &S, T *ext, int64_t klo, int64_t khi, int lane) {
        const float2 an = to_df(exp_from_tables(S.E, klo));
        for (int64_t kp = klo + lane; kp <= khi; kp += 32) {
            const float2 u = S.updf[kp - klo];
            float h, l, rh, rl;
            fft::df_mul(an.x, an.y, u.x, u.y, h, l);
            if (S.P.model == AOP_BSM_PUT) fft::df_add(1.0f, 0.0f, -h, -l, rh, rl);
            else fft::df_add(h, l, -S.kdf.x, -S.kdf.y, rh, rl);
            ext[kp - klo] = make_float2(rh, rl);
        }
    }
    __device__ static float2 to_df(double v) {
        const float h = (float)v;
        return make_float2(h, (float)(v - (double)h));
    }
};

// Doubled-FP32 copies of the option's weights, K and powers of u.
__device__ inline float2 to_df(double v) { return ArithDF::to_df(v); }
__device__ void build_df_tables(Shared &S) {
    for (int j = threadIdx.x; j < kNaiveCap; j += blockDim.x) S.updf[j] = to_df(exp((double)j * S.P.logu));
    if (threadIdx.x < 3) S.wdf[threadIdx.x] = to_df(S.P.w[threadIdx.x]);
    if (threadIdx.x == 3) S.kdf = to_df(S.P.K);
}

// ------------------------------------------------------------ the walker
template <int MODE, bool HELP = false>
struct Walker {
    using V = typename fft::Cx<MODE>::V;
    Cta<MODE> &c;
    Shared &S;
    const Params &P;
    const ExpTables &E;
    double *exw;                  // exercise values of the current base case
    int32_t *bnd;
    Counters &cnt;
    int lane;
    double *gk;                   // delta, gamma, theta of this option (nullable)

    __device__ Walker(Cta<MODE> &c_, double *buf, int32_t *bnd_, Counters &cnt_, double *gk_ = nullptr)
        : c(c_), S(c_.S), P(c_.S.P), E(c_.S.E), exw(buf),
          bnd(bnd_), cnt(cnt_),
          lane(threadIdx.x & 31), gk(gk_) {}

    __device__ void record(int64_t row, int32_t v) const {
        if (bnd && lane == 0) bnd[row] = v;
    }
    __device__ void record_range(int64_t r0, int64_t r1, int32_t v) const {
        if (!bnd) return;
        for (int64_t r = r0 + lane; r <= r1; r += 32) bnd[r] = v;
    }

    // post a linear advance into the slot of depth d
    __device__ void post(int d, const Buf &in, int64_t x_lo, int64_t x_hi, const Buf &out, int64_t g) {
        if constexpr (HELP) {
            int lgN = ilog2_ceil(x_hi - x_lo + 1);
            lgN = lgN < 2 ? 2 : lgN;
            if (c.help_lg() && lgN >= c.help_lg()) {
                // on the board: the input rows this warp wrote become visible
                // to every SM before the task word does
                __threadfence();
                __syncwarp();
                if (lane == 0) {
                    Board *bd = c.board();
                    GTask &t = bd->t[d];
                    t.in = in;
                    t.out = out;
                    t.x_lo = x_lo;
                    t.x_hi = x_hi;
                    t.g = g;
                    t.lgN = lgN;
                    t.err = 0;
                    t.posted_ns = gtime();
                    __threadfence();
                    atomicExch(&t.word, gword(S.gen, TASK_POSTED));
                    atomicOr(&bd->mask, 1u << d);
                    S.tasks[d].state = TASK_BOARD;
                }
                __syncwarp();
                return;
            }
        }
        if (lane == 0) {
            Task &t = S.tasks[d];
            t.in = in;
            t.out = out;
            t.x_lo = x_lo;
            t.x_hi = x_hi;
            t.g = g;
            int lgN = ilog2_ceil(x_hi - x_lo + 1);
            t.lgN = lgN < 2 ? 2 : lgN;
            __threadfence_block();
            t.state = TASK_POSTED;
            atomicOr((unsigned *)&S.posted, 1u << d);
        }
        __syncwarp();
    }
    // wait until the task of depth d is done (if one is outstanding)
    __device__ void wait(int d) {
        if (lane == 0) {
            Task &t = S.tasks[d];
            const uint64_t t0 = gtime();
            unsigned ns = 16;            // backoff: a long wait polls less often
            const uint64_t lim = wait_limit(c.a);
            if (HELP && t.state == TASK_BOARD) {
                GTask &gt = c.board()->t[d];
                const unsigned long long done = gword(S.gen, TASK_DONE);
                while (*(volatile unsigned long long *)&gt.word != done) {
                    __nanosleep(ns);
                    if (ns < 256) ns <<= 1;
                    if (gtime() - t0 > lim) { atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT); break; }
                }
                __threadfence();         // the output rows, written on another SM, are seen from here on
                if (gt.err) atomicCAS((int *)&S.err, 0, gt.err);
                if (*(volatile unsigned long long *)&gt.word == done) gt.word = gword(S.gen, TASK_FREE);
            } else {
                while (t.state == TASK_POSTED || t.state == TASK_CLAIMED) {
                    __nanosleep(ns);
                    if (ns < 128) ns <<= 1;
                    if (gtime() - t0 > lim) { atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT); break; }
                }
            }
            cnt.wait_ns += (long long)(gtime() - t0);
            t.state = TASK_FREE;
            __threadfence_block();
        }
        __syncwarp();
    }

    // ----- base cases (values in registers, exercise table in shared memory)

    __device__ int64_t naive_call(int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf &in, const Buf &out) {
        const uint64_t tb0 = gtime();
        const int64_t r = naive_call_body(i0, c0, b, h, in, out);
        if (lane == 0) {
            cnt.base_ns += (long long)(gtime() - tb0);
            cnt.base_calls++;
            cnt.base_rows += h;
        }
        return r;
    }
    // Row values live in registers: lane l holds cells t = x - c0 = l + 32 r,
    // r < R, updated in place (ascending r, so the right neighbours a lane
    // reads by shuffle are still the previous row's).  Every cell of the window
    // takes max(continuation, exercise) (Def. 2.1) from lane-local operands:
    // its exercise value comes from the base case's table at an address that
    // does not depend on the values, so no value waits for the divider.  The cells right of the top row's divider
    // tb stay green in every row below (Cor. 2.7) and hold their exercise
    // values, which closes the window on the right.  A row's divider (the last
    // real cell whose continuation is at least its exercise value) comes from
    // one ballot per register: a row costs one shuffle, one stencil sum, one
    // max and the ballots (lattice cells past a row's end, D i, get values
    // that only such cells read).  A is the arithmetic (FP64, or doubled FP32 on the FP32 pipe).
    template <int R, int D, class A>
    __device__ int64_t call_rows(int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf &in, const Buf &out,
                                 int64_t klo, int64_t khi) {
        using T = typename A::T;
        const typename A::Wts w = A::weights(S);
        const T *ext = (const T *)exw;
        // 32-bit arithmetic relative to (i0, c0) inside the base case: column
        // t = x - c0, row offset k = i0 - i.  The exercise value of (k, t)
        // sits at slot sbase + alpha t + k of the table, clamped into it (the
        // cells that can reach the clamp are past the window or the rows).
        const int alpha = (P.model == AOP_BINOMIAL_CALL) ? 2 : 1;
        const int sbase = (int)(alpha * c0 - i0 + P.T - klo);
        const int kmax = (int)(khi - klo);
        const int clip0 = (int)((int64_t)D * i0 - c0);   // row i0 - k ends at column clip0 - D k
        const int hh = (int)h;
        const int tb = (int)(b - c0);
        int32_t *const rec = (lane == 0 && bnd) ? bnd + i0 : nullptr;   // rec[-k] = row i0 - k
        auto slot = [&](int k, int t) { return min(max(sbase + alpha * t + k, 0), kmax); };
        T val[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int t = lane + 32 * r;
            val[r] = A::zero();
            if (t <= tb) val[r] = A::template load<MODE>(in, c0 + t);
            else if (t <= tb + D) val[r] = ext[slot(0, t)];
        }
        int bn = tb;
        long long cells = 0;
        const long long lc0 = clock64();
        for (int k = 1; k <= hh; k++) {
            const int lim = min(tb, clip0 - D * k);   // last real cell of the window in this row
            const int bprev = bn;
            int nbn = -1;
            // straight-line over the registers (R fits the window), so that
            // their shuffles, sums and maxima overlap
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int t = lane + 32 * r;
                const T ex = ext[slot(k, t)];      // independent of the values: issued early
                const T nx = (r + 1 < R) ? val[(r + 1) % R] : A::zero();
                const T n1 = A::shfl(lane == 0 ? nx : val[r], (lane + 1) & 31);
                T cont;
                if (D == 2) {
                    const T n2 = A::shfl(lane <= 1 ? nx : val[r], (lane + 2) & 31);
                    cont = A::dot3(w, val[r], n1, n2);
                } else {
                    cont = A::dot2(w, val[r], n1);
                }
                const bool red = A::cont_ge(cont, ex);
                val[r] = (red && t <= tb) ? cont : ex;
                // bit l: cell l + 32 r is a red cell of the row
                const unsigned bl = __ballot_sync(0xffffffffu, red && t <= lim);
                if (bl) nbn = 32 * r + 31 - __clz(bl);
            }
            // the previous row's divider is stored now, after this row's
            // shuffles, so that the store does not hold them back
            if (k > 1 && rec) rec[-(k - 1)] = (int32_t)(c0 + bprev);
            bn = nbn;
            cells += max(lim + 1, 0);
        }
        if (hh >= 1 && rec) rec[-hh] = (int32_t)(c0 + bn);
        if (lane == 0) cnt.loop_cyc += clock64() - lc0;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int t = lane + 32 * r;
            if (t <= bn) A::template store<MODE>(out, c0 + t, val[r]);
        }
        if (lane == 0) cnt.base_cells += cells;
        return c0 + bn;
    }

    // Doubled-FP32 rows with each lane holding R contiguous cells t = R l + c:
    // a row needs only the D cells right of a lane's last cell, from the next
    // lane (D shuffles of a pair); each cell carries its node price, multiplied
    // by u once per row (moving down a row raises the price exponent by one),
    // and its exercise value is that price less K; the divider is one maximum
    // over the lanes.  The cells and their values are those of call_rows: every
    // cell takes max(continuation, exercise) (Def. 2.1), the cells right of
    // the top row's divider stay green (Cor. 2.7).  The price recurrence adds
    // at most a few units of 2^-48 relative a row over the <= 64 rows of a
    // base case.
    template <int R, int D>
    __device__ int64_t call_rows_df(int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf &in, const Buf &out,
                                    int64_t klo) {
        using A = ArithDF;
        const A::Wts w = A::weights(S);
        const int alpha = (P.model == AOP_BINOMIAL_CALL) ? 2 : 1;
        const int sbase = (int)(alpha * c0 - i0 + P.T - klo);   // u-table slot of cell (0, t): sbase + alpha t
        const int clip0 = (int)((int64_t)D * i0 - c0);         // row i0 - k ends at column clip0 - D k
        const int hh = (int)h;
        const int tb = (int)(b - c0);
        int32_t *const rec = (lane == 0 && bnd) ? bnd + i0 : nullptr;   // rec[-k] = row i0 - k
        const float2 an = to_df(exp_from_tables(E, klo));      // node price of exponent index klo
        const float2 u = S.updf[1];
        const float2 K = S.kdf;
        float2 val[R], px[R];
#pragma unroll
        for (int c = 0; c < R; c++) {
            const int t = R * lane + c;
            const float2 g = S.updf[min(max(sbase + alpha * t, 0), kNaiveCap - 1)];
            fft::df_mul(an.x, an.y, g.x, g.y, px[c].x, px[c].y);
            float2 e0;
            fft::df_add(px[c].x, px[c].y, -K.x, -K.y, e0.x, e0.y);
            val[c] = A::zero();
            if (t <= tb) val[c] = A::template load<MODE>(in, c0 + t);
            else if (t <= tb + D) val[c] = e0;
        }
        int bn = tb;
        long long cells = 0;
        const long long lc0 = clock64();
        for (int k = 1; k <= hh; k++) {
            const int lim = min(tb, clip0 - D * k);   // last real cell of the window in this row
            const int bprev = bn;
            const float2 s1 = A::shfl(val[0], (lane + 1) & 31);
            float2 s2 = A::zero();
            if (D == 2) s2 = (R == 1) ? A::shfl(val[0], (lane + 2) & 31) : A::shfl(val[R > 1 ? 1 : 0], (lane + 1) & 31);
            int last = -1;
#pragma unroll
            for (int c = 0; c < R; c++) {
                const int t = R * lane + c;
                const float2 a1 = (c + 1 < R) ? val[(c + 1) % R] : s1;
                float2 cont;
                if (D == 2) {
                    const float2 a2 = (c + 2 < R) ? val[(c + 2) % R] : ((c + 2 == R) ? s1 : s2);
                    cont = A::dot3(w, val[c], a1, a2);
                } else {
                    cont = A::dot2(w, val[c], a1);
                }
                fft::df_mul(px[c].x, px[c].y, u.x, u.y, px[c].x, px[c].y);
                float2 ex;
                fft::df_add(px[c].x, px[c].y, -K.x, -K.y, ex.x, ex.y);
                const bool red = A::cont_ge(cont, ex);
                val[c] = (red && t <= tb) ? cont : ex;
                if (red && t <= lim) last = t;
            }
            const int nbn = __reduce_max_sync(0xffffffffu, last);
            // the previous row's divider is stored after this row's shuffles
            if (k > 1 && rec) rec[-(k - 1)] = (int32_t)(c0 + bprev);
            bn = nbn;
            cells += max(lim + 1, 0);
        }
        if (hh >= 1 && rec) rec[-hh] = (int32_t)(c0 + bn);
        if (lane == 0) cnt.loop_cyc += clock64() - lc0;
#pragma unroll
        for (int c = 0; c < R; c++) {
            const int t = R * lane + c;
            if (t <= bn) A::template store<MODE>(out, c0 + t, val[c]);
        }
        if (lane == 0) cnt.base_cells += cells;
        return c0 + bn;
    }

    template <class A>
    __device__ int64_t call_dispatch(int64_t need, int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf &in,
                                     const Buf &out, int64_t klo, int64_t khi) {
        if (std::is_same<A, ArithDF>::value) {   // no table: prices carried in registers
            if (P.D == 1) {
                if (need <= 32) return call_rows_df<1, 1>(i0, c0, b, h, in, out, klo);
                if (need <= 64) return call_rows_df<2, 1>(i0, c0, b, h, in, out, klo);
                if (need <= 128) return call_rows_df<4, 1>(i0, c0, b, h, in, out, klo);
                return call_rows_df<8, 1>(i0, c0, b, h, in, out, klo);
            }
            if (need <= 32) return call_rows_df<1, 2>(i0, c0, b, h, in, out, klo);
            if (need <= 64) return call_rows_df<2, 2>(i0, c0, b, h, in, out, klo);
            if (need <= 128) return call_rows_df<4, 2>(i0, c0, b, h, in, out, klo);
            return call_rows_df<8, 2>(i0, c0, b, h, in, out, klo);
        }
        const long long fc0 = clock64();
        A::fill(S, (typename A::T *)exw, klo, khi, lane);
        __syncwarp();
        if (lane == 0) cnt.fill_cyc += clock64() - fc0;
        if (P.D == 1) {
            if (need <= 32) return call_rows<1, 1, A>(i0, c0, b, h, in, out, klo, khi);
            if (need <= 64) return call_rows<2, 1, A>(i0, c0, b, h, in, out, klo, khi);
            if (need <= 128) return call_rows<4, 1, A>(i0, c0, b, h, in, out, klo, khi);
            return call_rows<8, 1, A>(i0, c0, b, h, in, out, klo, khi);
        }
        if (need <= 32) return call_rows<1, 2, A>(i0, c0, b, h, in, out, klo, khi);
        if (need <= 64) return call_rows<2, 2, A>(i0, c0, b, h, in, out, klo, khi);
        if (need <= 128) return call_rows<4, 2, A>(i0, c0, b, h, in, out, klo, khi);
        return call_rows<8, 2, A>(i0, c0, b, h, in, out, klo, khi);
    }

    __device__ int64_t naive_call_body(int64_t i0, int64_t c0, int64_t b, int64_t h, const Buf &in, const Buf &out) {
        const int D = P.D;
        const int64_t need = b - c0 + 1 + D;
        // exercise values the base case can touch (the divider moves <= 1 cell
        // per row): one table of exponent indices, filled once
        const int64_t klo = max((int64_t)0, ex_index(P, i0, c0) - 2);
        const int64_t khi = min(2 * P.T, ex_index(P, i0 - h, b + D) + 2);
        if (need > kRegCells || khi - klo + 1 > kNaiveCap) {   // never expected
            if (lane == 0) atomicCAS((int *)&S.err, 0, AOP_EINTERNAL);
            return b;
        }
        int64_t r;
        if (MODE == 0 || (double)(khi - klo) * P.logu > kDfLogRange)
            r = call_dispatch<ArithF64>(need, i0, c0, b, h, in, out, klo, khi);
        else
            r = call_dispatch<ArithDF>(need, i0, c0, b, h, in, out, klo, khi);
        __threadfence_block();
        __syncwarp();
        return r;
    }

    __device__ int64_t naive_put(int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h, const Buf &in,
                                 const Buf &out) {
        const uint64_t tb0 = gtime();
        const int64_t r = naive_put_body(n, lo, hi, f, h, in, out);
        if (lane == 0) {
            cnt.base_ns += (long long)(gtime() - tb0);
            cnt.base_calls++;
            cnt.base_rows += h;
        }
        return r;
    }
    // Put rows in registers (lane l holds cells x = lo + l + 32 r), updated
    // in place in ascending r (each lane keeps its old value of the register
    // below for the left neighbour of lane 0).  The window shrinks by one cell
    // per side per row.  Every cell takes max(continuation, exercise)
    // (Def. 2.1 for the put) from lane-local operands; the put's exercise
    // value does not depend on the time step, so each lane holds its cells'
    // values for the whole base case.  A row's divider (the last cell of the
    // row whose exercise value exceeds its continuation) comes from one ballot
    // per register.
    template <int R, class A>
    __device__ int64_t put_rows(int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h, const Buf &in,
                                const Buf &out) {
        using T = typename A::T;
        const typename A::Wts w = A::weights(S);
        const T *ext = (const T *)exw;
        const int span = (int)(hi - lo);          // window cells 0 .. span
        const int fl = (int)(f - lo);             // divider of row n, relative to lo
        T val[R], ex[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int t = lane + 32 * r;
            ex[r] = ext[min(t, span)];
            val[r] = A::zero();
            if (t <= span) val[r] = (t <= fl) ? ex[r] : A::template load<MODE>(in, lo + t);
        }
        int32_t *const rec = (lane == 0) ? bnd : nullptr;
        const int hh = (int)h;
        int fn = fl;
        long long cells = 0;
        for (int k = 1; k <= hh; k++) {
            const int fprev = fn;
            int nfn = k - 1;                      // none: left of this row's window
            T prev = A::zero();
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int t = lane + 32 * r;
                const T nx = (r + 1 < R) ? val[(r + 1) % R] : A::zero();
                const T vl = A::shfl(lane == 31 ? prev : val[r], (lane + 31) & 31);
                const T vr = A::shfl(lane == 0 ? nx : val[r], (lane + 1) & 31);
                const T cv = A::dot3(w, vl, val[r], vr);
                prev = val[r];
                const bool green = A::ex_gt(ex[r], cv);
                val[r] = green ? ex[r] : cv;
                // bit l: cell l + 32 r is a green cell of the row
                const unsigned bl = __ballot_sync(0xffffffffu, green && t >= k && t <= span - k);
                if (bl) nfn = 32 * r + 31 - __clz(bl);
            }
            // the previous row's divider is stored after this row's shuffles
            if (k > 1 && rec)
                rec[n + k - 1] = (fprev >= k - 1) ? (int32_t)(lo + fprev) : (int32_t)AOP_BOUNDARY_NONE_PUT;
            fn = nfn;
            cells += span - 2 * k + 1;
        }
        if (hh >= 1 && rec) rec[n + hh] = (fn >= hh) ? (int32_t)(lo + fn) : (int32_t)AOP_BOUNDARY_NONE_PUT;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int t = lane + 32 * r;
            if (t >= max(hh, fn + 1) && t <= span - hh) A::template store<MODE>(out, lo + t, val[r]);
        }
        if (lane == 0) cnt.base_cells += cells;
        return lo + fn;
    }

    // Doubled-FP32 put rows with each lane holding R contiguous cells
    // t = R l + c of the window (t = x - lo): a row needs the cell left of a
    // lane's first cell and the one right of its last, from the neighbouring
    // lanes (two shuffles of a pair); the exercise values (which for the put
    // do not depend on the time step) stay in registers; every cell takes
    // max(continuation, exercise) (Def. 2.1 for the put) and the divider -- the
    // last cell of the row whose exercise value exceeds its continuation -- is
    // one maximum over the lanes.  The cells and values are those of put_rows.
    template <int R>
    __device__ int64_t put_rows_df(int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h, const Buf &in,
                                   const Buf &out) {
        using A = ArithDF;
        const A::Wts w = A::weights(S);
        const float2 *ext = (const float2 *)exw;
        const int span = (int)(hi - lo);          // window cells 0 .. span
        const int fl = (int)(f - lo);             // divider of row n, relative to lo
        float2 val[R], ex[R];
#pragma unroll
        for (int c = 0; c < R; c++) {
            const int t = R * lane + c;
            ex[c] = ext[min(t, span)];
            val[c] = A::zero();
            if (t <= span) val[c] = (t <= fl) ? ex[c] : A::template load<MODE>(in, lo + t);
        }
        int32_t *const rec = (lane == 0) ? bnd : nullptr;
        const int hh = (int)h;
        int fn = fl;
        long long cells = 0;
        for (int k = 1; k <= hh; k++) {
            const int fprev = fn;
            const float2 left = A::shfl(val[R - 1], (lane + 31) & 31);
            const float2 right = A::shfl(val[0], (lane + 1) & 31);
            float2 prev = left;
            int last = -1;
#pragma unroll
            for (int c = 0; c < R; c++) {
                const int t = R * lane + c;
                const float2 nxt = (c + 1 < R) ? val[(c + 1) % R] : right;
                const float2 cv = A::dot3(w, prev, val[c], nxt);
                prev = val[c];
                const bool green = A::ex_gt(ex[c], cv);
                val[c] = green ? ex[c] : cv;
                if (green && t >= k && t <= span - k) last = t;
            }
            const int m = __reduce_max_sync(0xffffffffu, last);
            // the previous row's divider is stored after this row's shuffles
            if (k > 1 && rec)
                rec[n + k - 1] = (fprev >= k - 1) ? (int32_t)(lo + fprev) : (int32_t)AOP_BOUNDARY_NONE_PUT;
            fn = (m >= k) ? m : k - 1;            // none: left of this row's window
            cells += span - 2 * k + 1;
        }
        if (hh >= 1 && rec) rec[n + hh] = (fn >= hh) ? (int32_t)(lo + fn) : (int32_t)AOP_BOUNDARY_NONE_PUT;
#pragma unroll
        for (int c = 0; c < R; c++) {
            const int t = R * lane + c;
            if (t >= max(hh, fn + 1) && t <= span - hh) A::template store<MODE>(out, lo + t, val[c]);
        }
        if (lane == 0) cnt.base_cells += cells;
        return lo + fn;
    }

    template <class A>
    __device__ int64_t put_dispatch(int64_t w, int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h,
                                    const Buf &in, const Buf &out) {
        A::fill(S, (typename A::T *)exw, ex_index(P, n, lo), ex_index(P, n, hi), lane);
        __syncwarp();
        if (std::is_same<A, ArithDF>::value) {
            if (w <= 32) return put_rows_df<1>(n, lo, hi, f, h, in, out);
            if (w <= 64) return put_rows_df<2>(n, lo, hi, f, h, in, out);
            if (w <= 128) return put_rows_df<4>(n, lo, hi, f, h, in, out);
            return put_rows_df<8>(n, lo, hi, f, h, in, out);
        }
        if (w <= 32) return put_rows<1, A>(n, lo, hi, f, h, in, out);
        if (w <= 64) return put_rows<2, A>(n, lo, hi, f, h, in, out);
        if (w <= 128) return put_rows<4, A>(n, lo, hi, f, h, in, out);
        return put_rows<8, A>(n, lo, hi, f, h, in, out);
    }

    __device__ int64_t naive_put_body(int64_t n, int64_t lo, int64_t hi, int64_t f, int64_t h, const Buf &in,
                                      const Buf &out) {
        const int64_t w = hi - lo + 1;
        if (w > kRegCells) {            // never expected: window wider than the registers
            if (lane == 0) atomicCAS((int *)&S.err, 0, AOP_EINTERNAL);
            return f;
        }
        int64_t r;
        if (MODE == 0 || (double)(hi - lo) * P.logu > kDfLogRange)
            r = put_dispatch<ArithF64>(w, n, lo, hi, f, h, in, out);
        else
            r = put_dispatch<ArithDF>(w, n, lo, hi, f, h, in, out);
        __threadfence_block();
        __syncwarp();
        return r;
    }

    // ----- call recursion (explicit stack; every lane holds the same state)
    struct FrameC {
        int64_t i0, c0, b, h;
        Buf in, out;
        int depth, phase, posted;
    };

    __device__ int64_t solve_call(int64_t i0, int64_t b, int64_t h, const Buf &row) {
        FrameC st[kMaxDepth];
        int sp = 0;
        int64_t ret = 0;
        const int D = P.D;
        st[sp++] = FrameC{i0, 0, b, h, row, row, 0, 0, 0};
        while (sp > 0) {
            if (S.err) return ret;
            FrameC &F = st[sp - 1];
            if (F.phase == 0) {
                if (F.b < F.c0) {
                    record_range(F.i0 - F.h, F.i0 - 1, (int32_t)(F.c0 - 1));
                    ret = F.c0 - 1;
                    sp--;
                    continue;
                }
                if ((F.h <= c.a.B && F.b - F.c0 + 1 + D <= kRegCells) || F.h < 2 || F.depth + 1 >= kMaxDepth) {
                    ret = naive_call(F.i0, F.c0, F.b, F.h, F.in, F.out);
                    sp--;
                    continue;
                }
                const int64_t h1 = F.h >> 1;
                const Buf M{c.mid(F.depth), F.c0};
                F.posted = 0;
                if (F.b - D * h1 >= F.c0) {
                    post(F.depth, F.in, F.c0, F.b, M, h1);
                    F.posted = 1;
                }
                const int64_t c1 = max(F.c0, F.b - D * h1 + 1);
                F.phase = 1;
                st[sp++] = FrameC{F.i0, c1, F.b, h1, F.in, M, F.depth + 1, 0, 0};
            } else if (F.phase == 1) {
                if (F.posted) wait(F.depth);
                const int64_t b1 = ret;
                const int64_t h1 = F.h >> 1, h2 = F.h - h1;
                const Buf M{c.mid(F.depth), F.c0};
                F.posted = 0;
                if (b1 - D * h2 >= F.c0) {
                    post(F.depth, M, F.c0, b1, F.out, h2);
                    F.posted = 1;
                }
                const int64_t c2 = max(F.c0, b1 - D * h2 + 1);
                F.phase = 2;
                st[sp++] = FrameC{F.i0 - h1, c2, b1, h2, M, F.out, F.depth + 1, 0, 0};
            } else {
                if (F.posted) wait(F.depth);
                sp--;
            }
        }
        return ret;
    }

    // ----- sensitivities from the rows next to the root
    // With gk set, the chain stops at row 2 of a call lattice (row T-2 of
    // the put grid) and the last two rows are evaluated here in FP64 from
    // that row's cells (red cells from the row buffer, green ones from the
    // exercise value), which keeps rows 1 and 2 for delta, gamma and theta.
    // The formulas are the standard lattice ones (centred differences on the
    // nodes of rows 1-2, the time step between row 0 and the middle node of
    // row 2 / row 1), in the option's own spot coordinates; a lattice put
    // priced as a mirrored call is mapped back cell by cell first
    // (put value = mirrored value times u^x, x the put node's exponent).
    __device__ double finish_call_greeks(int64_t b, const Buf &row) {
        const int D = P.D;
        double g2[5], g1[3], g0 = 0.0;
        int32_t b1 = -1, b0 = -1;
        if (lane == 0) {
            for (int j = 0; j <= 2 * D; j++)
                g2[j] = (j <= b) ? cell_ld<MODE>(row, j) : exercise(P, E, ex_index(P, 2, j));
            for (int j = 0; j <= D; j++) {
                double cv = P.w[0] * g2[j] + P.w[1] * g2[j + 1];
                if (D == 2) cv += P.w[2] * g2[j + 2];
                const double e = exercise(P, E, ex_index(P, 1, j));
                if (cv >= e) b1 = j;
                g1[j] = fmax(cv, e);
            }
            double cv = P.w[0] * g1[0] + P.w[1] * g1[1];
            if (D == 2) cv += P.w[2] * g1[2];
            const double e = exercise(P, E, ex_index(P, 0, 0));
            if (cv >= e) b0 = 0;
            g0 = fmax(cv, e);
            if (bnd) { bnd[1] = b1; bnd[0] = b0; }
            // option-side rows: o2[j], o1[j] with node price S0 u^{x(i, j)}
            const double u = exp(P.logu);
            const double S0 = P.mirror ? P.K : P.S;
            double o2[5], o1[3];
            for (int j = 0; j <= 2 * D; j++) {
                const int x = (D == 1) ? 2 * j - 2 : j - 2;
                o2[j] = P.mirror ? g2[2 * D - j] * exp(x * P.logu) : g2[j];
            }
            for (int j = 0; j <= D; j++) {
                const int x = (D == 1) ? 2 * j - 1 : j - 1;
                o1[j] = P.mirror ? g1[D - j] * exp(x * P.logu) : g1[j];
            }
            const double d = 1.0 / u;
            double delta, gamma, theta;
            if (D == 1) {
                delta = (o1[1] - o1[0]) / (S0 * (u - d));
                const double up = (o2[2] - o2[1]) / (S0 * (u * u - 1.0));
                const double dn = (o2[1] - o2[0]) / (S0 * (1.0 - d * d));
                gamma = (up - dn) / (0.5 * S0 * (u * u - d * d));
                theta = (o2[1] - g0) / (2.0 * P.dt);
            } else {
                delta = (o1[2] - o1[0]) / (S0 * (u - d));
                const double up = (o1[2] - o1[1]) / (S0 * (u - 1.0));
                const double dn = (o1[1] - o1[0]) / (S0 * (1.0 - d));
                gamma = (up - dn) / (0.5 * S0 * (u - d));
                theta = (o1[1] - g0) / P.dt;
            }
            gk[0] = delta; gk[1] = gamma; gk[2] = theta;
        }
        return __shfl_sync(0xffffffffu, g0, 0);
    }

    __device__ double finish_put_greeks(int64_t f, const Buf &row) {
        const int64_t T = P.T;
        double v2[5], v1[3], v0 = 0.0;
        int32_t f1 = AOP_BOUNDARY_NONE_PUT, f0 = AOP_BOUNDARY_NONE_PUT;
        if (lane == 0) {
            for (int k = -2; k <= 2; k++)
                v2[k + 2] = (k <= f) ? exercise(P, E, ex_index(P, T - 2, k)) : cell_ld<MODE>(row, k);
            for (int k = -1; k <= 1; k++) {
                const double cv = P.w[0] * v2[k + 1] + P.w[1] * v2[k + 2] + P.w[2] * v2[k + 3];
                const double e = exercise(P, E, ex_index(P, T - 1, k));
                if (e > cv) f1 = k;
                v1[k + 1] = fmax(cv, e);
            }
            const double cv = P.w[0] * v1[0] + P.w[1] * v1[1] + P.w[2] * v1[2];
            const double e = exercise(P, E, ex_index(P, T, 0));
            if (e > cv) f0 = 0;
            v0 = fmax(cv, e);
            if (bnd) { bnd[T - 1] = f1; bnd[T] = f0; }
            const double K = P.out_scale, S0 = P.S;
            const double up = exp(P.logu), dn = exp(-P.logu);
            const double delta = K * (v1[2] - v1[0]) / (S0 * (up - dn));
            const double gu = K * (v1[2] - v1[1]) / (S0 * (up - 1.0));
            const double gd = K * (v1[1] - v1[0]) / (S0 * (1.0 - dn));
            gk[0] = delta;
            gk[1] = (gu - gd) / (0.5 * S0 * (up - dn));
            gk[2] = K * (v1[1] - v0) / P.dt;
        }
        return P.out_scale * __shfl_sync(0xffffffffu, v0, 0);
    }

    __device__ double price_call(int64_t b) {
        const int D = P.D;
        const Buf row{(double *)(c.slot + c.a.off_r0), 0};
        const int64_t stop = gk ? 2 : 0;     // gk needs P.T >= 3
        int64_t i = P.T - 1;
        while (i > stop) {
            if (S.err) return __longlong_as_double(0x7ff8000000000000ll);
            if (b >= 0) {
                // a red value never exceeds its node price; transforms (sums
                // of up to 2^21 values) need it well inside the range: 1e30
                // for the FP32 cells, 1e300 in FP64
                const double sb = exercise(P, E, ex_index(P, i, b)) + P.K;
                if (!(sb < (MODE == 0 ? 1e300 : 1e30))) {
                    if (lane == 0) atomicCAS((int *)&S.err, 0, AOP_ERANGE);
                    return __longlong_as_double(0x7ff8000000000000ll);
                }
            }
            if (b < 0) {                     // rows 0 .. i are green
                record_range(0, i - 1, -1);
                if (gk) return finish_call_greeks(-1, row);
                return exercise(P, E, ex_index(P, 0, 0));
            }
            const int64_t avail = i - kLeftoverCall;
            if (avail < c.a.B) {
                b = naive_call(i, 0, b, i - stop, row, row);
                i = stop;
                break;
            }
            const int64_t w = b + 1;
            const int64_t want = max((int64_t)c.a.B, (w + D - 1) / D);
            int64_t h = c.a.B;
            while (2 * h <= want && 2 * h <= avail) h *= 2;
            b = solve_call(i, b, h, row);
            i -= h;
        }
        if (gk) return S.err ? 0.0 : finish_call_greeks(b, row);
        if (b < 0) return exercise(P, E, ex_index(P, 0, 0));
        return cell_ld<MODE>(row, 0);
    }

    // ----- put recursion
    struct FrameP {
        int64_t n, lo, hi, f, h;
        Buf in, out;
        int depth, phase, posted;
    };

    __device__ int64_t solve_put(int64_t n0, int64_t lo0, int64_t hi0, int64_t f0, int64_t h0, const Buf &row) {
        FrameP st[kMaxDepth];
        int sp = 0;
        int64_t ret = 0;
        st[sp++] = FrameP{n0, lo0, hi0, f0, h0, row, row, 0, 0, 0};
        while (sp > 0) {
            if (S.err) return ret;
            FrameP &F = st[sp - 1];
            const int64_t h1 = F.h >> 1, h2 = F.h - h1;
            if (F.phase == 0) {
                if (F.f < F.lo) {        // no green cell in the window: one advance
                    post(F.depth, F.in, F.lo, F.hi, F.out, F.h);
                    record_range(F.n + 1, F.n + F.h, AOP_BOUNDARY_NONE_PUT);
                    wait(F.depth);
                    ret = F.lo + F.h - 1;
                    sp--;
                    continue;
                }
                if ((F.h <= c.a.Bput && F.hi - F.lo + 1 <= kRegCells) || F.h < 2 || F.depth + 1 >= kMaxDepth) {
                    ret = naive_put(F.n, F.lo, F.hi, F.f, F.h, F.in, F.out);
                    sp--;
                    continue;
                }
                const Buf M{c.mid(F.depth), F.lo + h1};
                F.posted = 0;
                if (F.f + 1 + h1 <= F.hi - h1) {
                    post(F.depth, F.in, F.f + 1, F.hi, M, h1);
                    F.posted = 1;
                }
                const int64_t lo2 = max(F.lo, F.f - 2 * h1), hi2 = min(F.hi, F.f + 2 * h1);
                F.phase = 1;
                st[sp++] = FrameP{F.n, lo2, hi2, F.f, h1, F.in, M, F.depth + 1, 0, 0};
            } else if (F.phase == 1) {
                if (F.posted) wait(F.depth);
                const int64_t f1 = ret;
                const int64_t lo1 = F.lo + h1, hi1 = F.hi - h1;
                const Buf M{c.mid(F.depth), lo1};
                if (f1 < lo1) {
                    post(F.depth, M, lo1, hi1, F.out, h2);
                    record_range(F.n + h1 + 1, F.n + F.h, AOP_BOUNDARY_NONE_PUT);
                    wait(F.depth);
                    ret = F.lo + F.h - 1;
                    sp--;
                    continue;
                }
                F.posted = 0;
                if (f1 + 1 + h2 <= hi1 - h2) {
                    post(F.depth, M, f1 + 1, hi1, F.out, h2);
                    F.posted = 1;
                }
                const int64_t lo2 = max(lo1, f1 - 2 * h2), hi2 = min(hi1, f1 + 2 * h2);
                F.phase = 2;
                st[sp++] = FrameP{F.n + h1, lo2, hi2, f1, h2, M, F.out, F.depth + 1, 0, 0};
            } else {
                if (F.posted) wait(F.depth);
                sp--;
            }
        }
        return ret;
    }

    __device__ double price_put(int64_t f) {
        const int64_t T = P.T;
        const Buf row{(double *)(c.slot + c.a.off_r0), -T};
        const int64_t stop = gk ? 2 : 0;     // gk needs T >= 3
        int64_t n = 1;
        while (T - n > stop) {
            if (S.err) return __longlong_as_double(0x7ff8000000000000ll);
            const int64_t R = T - n;
            if (f >= R) {                // every remaining cell is green
                if (bnd)
                    for (int64_t r = n + 1 + lane; r <= T; r += 32) bnd[r] = (int32_t)(T - r);
                if (gk) return finish_put_greeks(T, row);
                return P.out_scale * exercise(P, E, ex_index(P, T, 0));
            }
            if (R < 2 * c.a.Bput) {
                f = naive_put(n, -R, R, f, R - stop, row, row);
                n = T - stop;
                break;
            }
            int64_t h = c.a.Bput;
            while (2 * h <= R / 2) h *= 2;
            f = solve_put(n, -R, R, f, h, row);
            n += h;
        }
        if (gk) return S.err ? 0.0 : finish_put_greeks(f, row);
        if (f >= 0) return P.out_scale * exercise(P, E, ex_index(P, T, 0));
        return P.out_scale * cell_ld<MODE>(row, 0);
    }
};

// -------------------------------------------------- block-level first rows
// Calls: row T (continuation 0) and row T-1 over the whole row.  Cor. 2.7
// holds from row T-1 down only: with r > q the divider jumps right between
// rows T and T-1.  Returns the divider of row T-1.
template <int MODE>
__device__ int64_t first_rows_call(Cta<MODE> &c, int32_t *bnd) {
    Shared &S = c.S;
    const Params &P = S.P;
    const ExpTables &E = S.E;
    const int64_t T = P.T;
    const int D = P.D;
    const Buf row{(double *)(c.slot + c.a.off_r0), 0};
    if (threadIdx.x == 0) S.bcast_i = -1;
    __syncthreads();
    int bt = -1;
    for (int64_t j = threadIdx.x; j <= (int64_t)D * T; j += blockDim.x)
        if (0.0 >= exercise(P, E, ex_index(P, T, j))) bt = max(bt, (int)j);
    bt = __reduce_max_sync(0xffffffffu, bt);
    if ((threadIdx.x & 31) == 0) atomicMax(&S.bcast_i, bt);
    __syncthreads();
    if (threadIdx.x == 0 && bnd) bnd[T] = S.bcast_i;
    __syncthreads();
    if (threadIdx.x == 0) S.bcast_i = -1;
    __syncthreads();
    const int64_t i = T - 1;
    int br = -1;
    const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
    for (int64_t j = threadIdx.x; j <= (int64_t)D * i; j += blockDim.x) {
        double cv = w0 * fmax(exercise(P, E, ex_index(P, T, j)), 0.0) +
                    w1 * fmax(exercise(P, E, ex_index(P, T, j + 1)), 0.0);
        if (D == 2) cv += w2 * fmax(exercise(P, E, ex_index(P, T, j + 2)), 0.0);
        cell_st<MODE>(row, j, cv);
        // Node prices beyond the FP64 range (e^709: long lattices at high
        // volatility) make both sides infinite; such cells lie far above any
        // early-exercise boundary and are left green (with no yield their
        // weight in the price is below the rounding of every other cell).
        const double e = exercise(P, E, ex_index(P, i, j));
        if (cv < INFINITY && e < INFINITY && cv >= e) br = max(br, (int)j);
    }
    br = __reduce_max_sync(0xffffffffu, br);
    if ((threadIdx.x & 31) == 0) atomicMax(&S.bcast_i, br);
    __syncthreads();
    const int64_t b = S.bcast_i;
    if (threadIdx.x == 0 && bnd) bnd[i] = (int32_t)b;
    __syncthreads();
    return b;
}

// Put: row 0 (the payoff) and row 1 over the whole row.  The BSM divider
// theorem's step k_n - k_{n+1} <= 1 rests on the divider cell being green by
// the max at row n; at the expiry row it is green by its payoff alone, so the
// step 0 -> 1 may move the divider arbitrarily far (r = 0: no cell stays
// green).  Returns the divider of row 1 (or -T-1 when it has no green cell).
template <int MODE>
__device__ int64_t first_rows_put(Cta<MODE> &c, int32_t *bnd) {
    Shared &S = c.S;
    const Params &P = S.P;
    const ExpTables &E = S.E;
    const int64_t T = P.T;
    const Buf row{(double *)(c.slot + c.a.off_r0), -T};
    if (threadIdx.x == 0) S.bcast_i = INT32_MIN;
    __syncthreads();
    int fb = INT32_MIN;
    for (int64_t k = -T + threadIdx.x; k <= T; k += blockDim.x)
        if (exercise(P, E, ex_index(P, 0, k)) > 0.0) fb = max(fb, (int)k);
    fb = __reduce_max_sync(0xffffffffu, fb);
    if ((threadIdx.x & 31) == 0) atomicMax(&S.bcast_i, fb);
    __syncthreads();
    if (threadIdx.x == 0 && bnd) bnd[0] = S.bcast_i;
    __syncthreads();
    if (threadIdx.x == 0) S.bcast_i = INT32_MIN;
    __syncthreads();
    // row 1 straight from the payoff max(e, 0) of row 0
    fb = INT32_MIN;
    const double wb = P.w[0], wc = P.w[1], wa = P.w[2];
    for (int64_t k = -(T - 1) + threadIdx.x; k <= T - 1; k += blockDim.x) {
        const double cv = wb * fmax(exercise(P, E, ex_index(P, 0, k - 1)), 0.0) +
                          wc * fmax(exercise(P, E, ex_index(P, 0, k)), 0.0) +
                          wa * fmax(exercise(P, E, ex_index(P, 0, k + 1)), 0.0);
        const double e = exercise(P, E, ex_index(P, 1, k));
        const bool green = e > cv;
        cell_st<MODE>(row, k, green ? e : cv);
        if (green) fb = max(fb, (int)k);
    }
    fb = __reduce_max_sync(0xffffffffu, fb);
    if ((threadIdx.x & 31) == 0) atomicMax(&S.bcast_i, fb);
    __syncthreads();
    const int f = S.bcast_i;
    if (threadIdx.x == 0 && bnd) bnd[1] = f;
    __syncthreads();
    return (f == INT32_MIN) ? -T - 1 : f;
}

// ------------------------------------------------------------------ kernel
// Helping CTA (warp 0): the next board with posted work, scanning the other
// CTAs' boards from this one's right neighbour on, 32 at a time.  Sets S.hk
// (-1: none now, -2: stop) and, for a board, the option, its generation and
// tilt, read between two equal reads of the generation.
template <int MODE>
__device__ void pick_board(const Cta<MODE> &c, Shared &S, int lane, uint64_t &hidle) {
    const DncArgs &a = c.a;
    int64_t k = -1;
    if (*(volatile int *)a.finished >= a.n) {
        k = -2;
    } else {
        for (int64_t base = 0; base < a.grid && k < 0; base += 32) {
            const int64_t i = base + lane;
            bool ok = false;
            if (i < a.grid - 1) {
                const Board *bd = c.board_of((blockIdx.x + 1 + i) % a.grid);
                ok = (bd->gen >> kGenBits) == a.epoch && *(const volatile unsigned *)&bd->mask != 0u &&
                     bd->opt >= 0;
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (m) k = (blockIdx.x + 1 + base + __ffs(m) - 1) % a.grid;
        }
    }
    if (lane == 0) {
        if (k >= 0) {
            const Board *bd = c.board_of(k);
            const unsigned long long g0 = bd->gen;
            __threadfence();
            const long long op = bd->opt;
            const int tl = bd->tilt;
            __threadfence();
            if (bd->gen != g0 || op < 0 || op >= a.n) {
                k = -1;
            } else {
                S.opt = (int)op;
                S.gen = g0;
                S.htilt = tl;
            }
        }
        const uint64_t now = gtime();
        if (k >= 0) hidle = now;
        else if (k == -1 && now - hidle > kHelpIdleNs) k = -2;   // nothing to help for a while: stop
        S.hk = (int)k;
    }
    __syncwarp();
}

// HELP: batch launches whose CTAs help one another (board tasks, helping
// sessions); without it, the plain kernel of serving sessions, of the
// FP32-split mode and of launches that ask for no helping.
template <int MODE, bool HELP>
__global__ void __launch_bounds__(Shape<MODE>::threads, Shape<MODE>::min_ctas)
dnc_kernel(const __grid_constant__ DncArgs a)
{
    using V = typename fft::Cx<MODE>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *walker_buf = (double *)smem_raw;                              // kNaiveCap doubles
    V *tiles = (V *)(smem_raw + kNaiveCap * sizeof(double));            // one tile per worker
    char *slot = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    Cta<MODE> c(a, S, slot);
    Counters cnt{};
    // Place the recursion warp of each resident CTA on a different SM
    // sub-partition: FP64 instructions issue at a fraction of a warp per cycle
    // per sub-partition, and the walkers' FP64 base cases must not queue behind
    // one another.  The k-th CTA to arrive on an SM walks with the warp whose
    // hardware slot lies in sub-partition k mod 4.
    __shared__ int s_walker;
    constexpr int kWarps = Shape<MODE>::warps;
    __shared__ int s_sub[kWarps];
    if (lane == 0) {
        unsigned wid_hw;
        asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid_hw));
        s_sub[warp] = (int)(wid_hw & 3);
    }
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        // FP64 mode: one walker per SM sub-partition (each issues its FP64
        // stencil on that partition's FP64 unit).  FP32 modes: all walkers on
        // sub-partition 0, so that no walker shares issue slots with the
        // convolution warps (AOP_FLAG_SPREAD_WALKERS: one per partition).
        const bool spread = (MODE == 0) || (a.flags & AOP_FLAG_SPREAD_WALKERS);
        s_walker = (spread && a.sm_slots) ? (atomicAdd(&a.sm_slots[smid & 1023], 1) & 3) : 0;
        S.helping = 0;
        S.hk = -1;
    }
    __syncthreads();
    int walker = 0;
    for (int w = 0; w < kWarps; w++)
        if (s_sub[w] == s_walker) { walker = w; break; }
    const int role = (warp - walker + kWarps) % kWarps;    // 0 = walker, 1.. = workers
    if constexpr (HELP) {
        if (c.help_lg() && threadIdx.x == 0) {
            // this launch's board: empty, stamped with the launch's epoch
            Board *bd = c.board();
            bd->opt = -1;
            bd->mask = 0;
            bd->helpers = 0;
            S.gen = (unsigned long long)a.epoch << kGenBits;
            for (int d = 0; d < kMaxDepth; d++) bd->t[d].word = gword(S.gen, TASK_FREE);
            __threadfence();
            bd->gen = S.gen;
        }
        uint64_t hidle = 0;          // (warp 0, lane 0) since when no board had work for this CTA
        for (;;) {
            if (warp == 0) {
                if (lane == 0) {
                    int64_t q = -1;
                    if (!S.helping) {
                        q = a.sreq ? claim_published(a) : atomicAdd(a.queue, 1);
                        if (!a.sreq && a.order && q < a.n) q = a.order[q];
                        if ((q < 0 || q >= a.n) && c.help_lg()) {
                            S.helping = 1;
                            hidle = gtime();
                        }
                    }
                    S.opt = q;
                }
                __syncwarp();
                if (S.helping) pick_board(c, S, lane, hidle);
            }
            __syncthreads();
            const bool own = !S.helping;
            const int64_t o = own ? S.opt : (S.hk >= 0 ? S.opt : -1);
            if (own && (o < 0 || o >= a.n)) break;
            if (!own && S.hk == -2) break;
            if (!own && S.hk < 0) {
                __syncthreads();     // every warp has read S.hk before warp 0 looks again
                __nanosleep(2000);   // no board has posted work
                continue;
            }
            if (threadIdx.x == 0) {
                if (!own) {
                    S.P = a.params[o];
                } else if (a.sreq) {
                    // fresh (uncached) loads of the request from host memory
                    static_assert(sizeof(aop_request) % 8 == 0, "request is whole 8-byte words");
                    aop_request rq;
                    const unsigned long long *src = (const unsigned long long *)&a.sreq[o];
                    unsigned long long *dst = (unsigned long long *)&rq;
                    for (int k = 0; k < (int)(sizeof(aop_request) / 8); k++) dst[k] = __ldcv(src + k);
                    S.P = make_params(rq);
                    if (S.P.status == AOP_OK && S.P.T > a.sT_max) S.P.status = AOP_EINVAL;
                } else {
                    S.P = a.params[o];
                }
                S.spec_n = 0;
                S.spec_lock = 0;
                for (int j = 0; j < kSpecLg * kSpecLg; j++) (&S.spec_map[0][0])[j] = 0;
                S.arena_used = 0;
                S.done = 0;
                S.err = 0;
                for (int d = 0; d < kMaxDepth; d++) S.tasks[d].state = TASK_FREE;
                S.posted = 0;
            }
            __syncthreads();
            if (own && S.P.status != AOP_OK) {
                if (threadIdx.x == 0) {
                    a.prices[o] = __longlong_as_double(0x7ff8000000000000ll);
                    if (a.sreq) {
                        a.status[o] = S.P.status;
                        __threadfence_system();
                        a.sdone[o] = 1;
                    }
                    if (a.finished) atomicAdd(a.finished, 1);
                }
                __syncthreads();
                continue;
            }
            uint64_t t_start = 0;
            if (threadIdx.x == 0 && a.opt_ns) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
            build_exp_tables(S.P, S.E);
            const bool may_tilt = S.P.model != AOP_BSM_PUT && S.P.kappa > 0.0 && !(a.flags & AOP_FLAG_TILT_OFF);
            if (may_tilt) build_tilt_tables<MODE>(S);
            __syncthreads();
            if (MODE != 0) build_df_tables(S);
            __syncthreads();
            int32_t *bnd = a.bnd ? a.bnd + a.bnd_off[o] : nullptr;
            const bool put = (S.P.model == AOP_BSM_PUT);
            int64_t first = 0;
            if (own) first = put ? first_rows_put(c, bnd) : first_rows_call(c, bnd);
            // Untilted, the rounding of every advance scales with the largest value
            // of its window (about S_b - K at the divider, node price S_b); tilted,
            // with the node price of each cell.  The FP32-split mode always tilts
            // calls (measured: 314 instead of 238 of the sweep's 455 priced options
            // within 1e-6); the FP64 and doubled modes, whose rounding is far below
            // the bounds, tilt when the continuation region reaches node prices far
            // above the strike (whole rows red, or S_b - K > 2 S0), where the
            // untilted window's range would swamp the cells near the money.
            c.tilt = false;
            if (!own) {
                c.tilt = S.htilt != 0;
            } else if (may_tilt) {
                const double sb = exercise(S.P, S.E, ex_index(S.P, S.P.T - 1, first)) + S.P.K;
                c.tilt = MODE == 1 || (a.flags & AOP_FLAG_TILT_ON) || first >= (int64_t)S.P.D * (S.P.T - 1) ||
                         sb - S.P.K > 2.0 * S.P.S;
            }
            if (own && c.help_lg()) {
                if (threadIdx.x == 0) {
                    // publish the option: helpers may take its board tasks from here on
                    Board *bd = c.board();
                    bd->opt = o;
                    bd->tilt = c.tilt ? 1 : 0;
                    S.gen++;
                    __threadfence();
                    bd->gen = S.gen;
                }
                __syncthreads();
            }
            double *gk = (a.greeks && S.P.T >= 3) ? a.greeks + 3 * o : nullptr;
            if (!own && threadIdx.x == 0) atomicAdd(&c.board_of(S.hk)->helpers, 1);
            if (MODE != 1 && !own && a.help_block) {
                // a CTA launched to help: one board advance at a time, all warps
                // on it.  The tile is a worker's, so the transform is split into
                // the same passes and stages as a worker's and the result is the
                // same to the bit.
                Board *bd = c.board_of(S.hk);
                uint64_t idle0 = gtime();
                for (;;) {
                    if (threadIdx.x == 0) {
                        int pick = -1;
                        if (bd->gen != S.gen) {
                            pick = -2;
                        } else if (!(a.flags & AOP_FLAG_TEST_STALL)) {
                            const unsigned long long want = gword(S.gen, TASK_POSTED);
                            unsigned m = *(volatile unsigned *)&bd->mask;
                            while (m) {
                                const int d = 31 - __clz(m);
                                m &= ~(1u << d);
                                if (atomicCAS(&bd->t[d].word, want, gword(S.gen, TASK_CLAIMED)) == want) {
                                    atomicAnd(&bd->mask, ~(1u << d));
                                    pick = d;
                                    break;
                                }
                            }
                        }
                        if (pick == -1 && gtime() - idle0 > kHelpIdleNs) pick = -2;
                        S.bcast_i = pick;
                    }
                    __syncthreads();
                    const int pick = S.bcast_i;
                    __syncthreads();
                    if (pick == -2) break;
                    if (pick < 0) {
                        __nanosleep(128);
                        continue;
                    }
                    __threadfence();         // the input rows, written on another SM, are seen from here on
                    const volatile GTask &g = bd->t[pick];
                    Task t;
                    t.in.p = g.in.p;
                    t.in.base = g.in.base;
                    t.out.p = g.out.p;
                    t.out.base = g.out.base;
                    t.x_lo = g.x_lo;
                    t.x_hi = g.x_hi;
                    t.g = g.g;
                    const uint64_t tb = gtime();
                    c.template conv<fft::BlockGroup, StoreCell<MODE>>(t.in, t.x_lo, t.x_hi, t.out, t.g, tiles,
                                                                      a.lg_tile, c.scratch(0), cnt);
                    __syncthreads();
                    const int err = S.err;
                    if (threadIdx.x == 0) {
                        GTask &gt = bd->t[pick];
                        if (err) gt.err = err;
                        __threadfence();     // the output rows before the word
                        atomicExch(&gt.word, gword(S.gen, TASK_DONE));
                        idle0 = gtime();
                        cnt.helped++;
                        cnt.helped_ns += (long long)(idle0 - tb);
                    }
                    if (err) break;
                }
            } else if (role == 0) {
                if (own) {
                    Walker<MODE, true> wk(c, walker_buf, bnd, cnt, gk);
                    const uint64_t tw0 = gtime();
                    const double price = put ? wk.price_put(first) : wk.price_call(first);
                    if (lane == 0) {
                        cnt.walker_ns += (long long)(gtime() - tw0);
                        S.price = price;
                        __threadfence_block();
                        S.done = 1;
                    }
                    __syncwarp();
                }
            } else {
                const int wid = role - 1;
                V *tile = tiles + ((int64_t)wid << a.lg_tile);
                // the board this worker takes multi-pass advances from (the CTA's
                // own, or the helped option's); only workers with global scratch
                Board *bd = (c.help_lg() && wid < Shape<MODE>::big) ? (own ? c.board() : c.board_of(S.hk)) : nullptr;
                const Board *hb = own ? nullptr : c.board_of(S.hk);
                uint64_t idle0 = gtime();
                unsigned nap = 32;           // idle backoff (ns), reset by each task
                for (;;) {
                    int pick = -1;           // depth of a local task, 32 + depth of a board task
                    if (lane == 0) {
                        if (own ? S.done != 0 : hb->gen != S.gen) pick = -2;
                        else if (!(a.flags & AOP_FLAG_TEST_STALL)) {
                            // posted slots from the mask word, deepest first
                            unsigned m = own ? S.posted : 0u;
                            while (m) {
                                const int d = 31 - __clz(m);
                                m &= ~(1u << d);
                                if (S.tasks[d].state != TASK_POSTED) continue;
                                if (wid >= Shape<MODE>::big && S.tasks[d].lgN > a.lg_tile) continue;
                                if (atomicCAS((int *)&S.tasks[d].state, TASK_POSTED, TASK_CLAIMED) == TASK_POSTED) {
                                    atomicAnd((unsigned *)&S.posted, ~(1u << d));
                                    pick = d;
                                    break;
                                }
                            }
                            if (pick < 0 && bd) {
                                const unsigned long long want = gword(S.gen, TASK_POSTED);
                                m = *(volatile unsigned *)&bd->mask;
                                // with helpers attached, the option's own workers
                                // take a board task only once it has waited
                                const bool defer = own && *(volatile int *)&bd->helpers > 0;
                                const uint64_t now = defer ? gtime() : 0;
                                while (m) {
                                    const int d = 31 - __clz(m);
                                    m &= ~(1u << d);
                                    if (defer && now - bd->t[d].posted_ns < kHelpDeferNs) continue;
                                    if (atomicCAS(&bd->t[d].word, want, gword(S.gen, TASK_CLAIMED)) == want) {
                                        atomicAnd(&bd->mask, ~(1u << d));
                                        pick = 32 + d;
                                        break;
                                    }
                                }
                            }
                        }
                    }
                    pick = __shfl_sync(0xffffffffu, pick, 0);
                    if (pick == -2) break;
                    if (pick < 0) {
                        __nanosleep(nap);
                        if (nap < 256) nap <<= 1;
                        if (gtime() - idle0 > (own ? wait_limit(a) : kHelpIdleNs)) {
                            if (own && lane == 0) atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT);
                            break;
                        }
                        continue;
                    }
                    const uint64_t tb = gtime();
                    Task t;
                    if (pick < 32) {
                        __threadfence_block();
                        t = *(const Task *)&S.tasks[pick];
                    } else {
                        __syncwarp();        // after lane 0's claim
                        __threadfence();     // the input rows, written on another SM, are seen from here on
                        const volatile GTask &g = bd->t[pick - 32];
                        t.in.p = g.in.p;
                        t.in.base = g.in.base;
                        t.out.p = g.out.p;
                        t.out.base = g.out.base;
                        t.x_lo = g.x_lo;
                        t.x_hi = g.x_hi;
                        t.g = g.g;
                    }
                    const int lgN = c.template conv<fft::WarpGroup, StoreCell<MODE>>(
                        t.in, t.x_lo, t.x_hi, t.out, t.g, tile, a.lg_tile, wid < Shape<MODE>::big ? c.scratch(wid) : nullptr,
                        cnt);
                    if (pick < 32) {
                        __threadfence_block();
                        __syncwarp();
                        if (lane == 0) S.tasks[pick].state = TASK_DONE;
                    } else {
                        __syncwarp();
                        if (lane == 0) {
                            GTask &g = bd->t[pick - 32];
                            if (S.err) g.err = S.err;
                            __threadfence();     // the output rows before the word
                            atomicExch(&g.word, gword(S.gen, TASK_DONE));
                        }
                        if (!own && S.err) break;
                    }
                    idle0 = gtime();
                    if (!own && lane == 0) {
                        cnt.helped++;
                        cnt.helped_ns += (long long)(idle0 - tb);
                    }
                    nap = 32;
                    if (lane == 0) {
                        cnt.busy_ns += (long long)(idle0 - tb);
                        cnt.hist_n[min(lgN, 23)]++;
                        cnt.hist_ns[min(lgN, 23)] += (long long)(idle0 - tb);
                    }
                }
            }
            __syncthreads();
            if (!own && threadIdx.x == 0) atomicSub(&c.board_of(S.hk)->helpers, 1);
            if (own && c.help_lg() && threadIdx.x == 0) {
                // end of the option on the board: revoke what no worker took, wait
                // for what helpers hold (their results land in this slot's rows),
                // then move the generation on so that helpers leave
                Board *bd = c.board();
                const unsigned long long g_end = S.gen + 1;
                for (int d = 0; d < kMaxDepth; d++) {
                    GTask &t = bd->t[d];
                    const unsigned long long w = atomicCAS(&t.word, gword(S.gen, TASK_POSTED), gword(g_end, TASK_FREE));
                    if (w != gword(S.gen, TASK_CLAIMED)) continue;
                    const uint64_t t0 = gtime();
                    while (*(volatile unsigned long long *)&t.word == w) {
                        __nanosleep(256);
                        if (gtime() - t0 > wait_limit(a)) { atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT); break; }
                    }
                    if (t.err) atomicCAS((int *)&S.err, 0, t.err);
                }
                bd->mask = 0;
                bd->opt = -1;
                S.gen = g_end;
                __threadfence();
                bd->gen = g_end;
            }
            if (own && threadIdx.x == 0) {
                const int err = S.err;
                a.prices[o] = err ? __longlong_as_double(0x7ff8000000000000ll) : S.price;
                if (a.greeks && (err || S.P.T < 3))
                    for (int g = 0; g < 3; g++) a.greeks[3 * o + g] = __longlong_as_double(0x7ff8000000000000ll);
                if (err) {
                    if (a.status) a.status[o] = err;
                    if (a.err) atomicCAS(a.err, 0, err);
                }
                if (a.opt_ns) {
                    uint64_t t_end;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                    a.opt_ns[o] = (int64_t)(t_end - t_start);
                }
                if (a.sreq) {
                    a.status[o] = err ? err : AOP_OK;
                    __threadfence_system();
                    a.sdone[o] = 1;
                }
                if (a.finished) atomicAdd(a.finished, 1);
            }
            if (!own && threadIdx.x == 0) hidle = gtime();   // idle time counts from the session's end
            __syncthreads();
        }
    } else {
        for (;;) {
            if (threadIdx.x == 0) {
                int64_t q = a.sreq ? claim_published(a) : atomicAdd(a.queue, 1);
                if (!a.sreq && a.order && q < a.n) q = a.order[q];
                S.opt = q;
            }
            __syncthreads();
            const int64_t o = S.opt;
            if (o < 0 || o >= a.n) break;
            if (threadIdx.x == 0) {
                if (a.sreq) {
                    // fresh (uncached) loads of the request from host memory
                    static_assert(sizeof(aop_request) % 8 == 0, "request is whole 8-byte words");
                    aop_request rq;
                    const unsigned long long *src = (const unsigned long long *)&a.sreq[o];
                    unsigned long long *dst = (unsigned long long *)&rq;
                    for (int k = 0; k < (int)(sizeof(aop_request) / 8); k++) dst[k] = __ldcv(src + k);
                    S.P = make_params(rq);
                    if (S.P.status == AOP_OK && S.P.T > a.sT_max) S.P.status = AOP_EINVAL;
                } else {
                    S.P = a.params[o];
                }
                S.spec_n = 0;
                S.spec_lock = 0;
                for (int j = 0; j < kSpecLg * kSpecLg; j++) (&S.spec_map[0][0])[j] = 0;
                S.arena_used = 0;
                S.done = 0;
                S.err = 0;
                for (int d = 0; d < kMaxDepth; d++) S.tasks[d].state = TASK_FREE;
                S.posted = 0;
            }
            __syncthreads();
            if (S.P.status != AOP_OK) {
                if (threadIdx.x == 0) {
                    a.prices[o] = __longlong_as_double(0x7ff8000000000000ll);
                    if (a.sreq) {
                        a.status[o] = S.P.status;
                        __threadfence_system();
                        a.sdone[o] = 1;
                    }
                }
                __syncthreads();
                continue;
            }
            uint64_t t_start = 0;
            if (threadIdx.x == 0 && a.opt_ns) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
            build_exp_tables(S.P, S.E);
            const bool may_tilt = S.P.model != AOP_BSM_PUT && S.P.kappa > 0.0 && !(a.flags & AOP_FLAG_TILT_OFF);
            if (may_tilt) build_tilt_tables<MODE>(S);
            __syncthreads();
            if (MODE != 0) build_df_tables(S);
            __syncthreads();
            int32_t *bnd = a.bnd ? a.bnd + a.bnd_off[o] : nullptr;
            const bool put = (S.P.model == AOP_BSM_PUT);
            const int64_t first = put ? first_rows_put(c, bnd) : first_rows_call(c, bnd);
            // Untilted, the rounding of every advance scales with the largest value
            // of its window (about S_b - K at the divider, node price S_b); tilted,
            // with the node price of each cell.  The FP32-split mode always tilts
            // calls (measured: 314 instead of 238 of the sweep's 455 priced options
            // within 1e-6); the FP64 and doubled modes, whose rounding is far below
            // the bounds, tilt when the continuation region reaches node prices far
            // above the strike (whole rows red, or S_b - K > 2 S0), where the
            // untilted window's range would swamp the cells near the money.
            c.tilt = false;
            if (may_tilt) {
                const double sb = exercise(S.P, S.E, ex_index(S.P, S.P.T - 1, first)) + S.P.K;
                c.tilt = MODE == 1 || (a.flags & AOP_FLAG_TILT_ON) || first >= (int64_t)S.P.D * (S.P.T - 1) ||
                         sb - S.P.K > 2.0 * S.P.S;
            }
            double *gk = (a.greeks && S.P.T >= 3) ? a.greeks + 3 * o : nullptr;
            if (role == 0) {
                Walker<MODE> wk(c, walker_buf, bnd, cnt, gk);
                const uint64_t tw0 = gtime();
                const double price = put ? wk.price_put(first) : wk.price_call(first);
                if (lane == 0) {
                    cnt.walker_ns += (long long)(gtime() - tw0);
                    S.price = price;
                    __threadfence_block();
                    S.done = 1;
                }
                __syncwarp();
            } else {
                const int wid = role - 1;
                V *tile = tiles + ((int64_t)wid << a.lg_tile);
                uint64_t idle0 = gtime();
                unsigned nap = 32;           // idle backoff (ns), reset by each task
                for (;;) {
                    int pick = -1;
                    if (lane == 0) {
                        if (S.done) pick = -2;
                        else if (!(a.flags & AOP_FLAG_TEST_STALL)) {
                            // posted slots from the mask word, deepest first
                            unsigned m = S.posted;
                            while (m) {
                                const int d = 31 - __clz(m);
                                m &= ~(1u << d);
                                if (S.tasks[d].state != TASK_POSTED) continue;
                                if (wid >= Shape<MODE>::big && S.tasks[d].lgN > a.lg_tile) continue;
                                if (atomicCAS((int *)&S.tasks[d].state, TASK_POSTED, TASK_CLAIMED) == TASK_POSTED) {
                                    atomicAnd((unsigned *)&S.posted, ~(1u << d));
                                    pick = d;
                                    break;
                                }
                            }
                        }
                    }
                    pick = __shfl_sync(0xffffffffu, pick, 0);
                    if (pick == -2) break;
                    if (pick < 0) {
                        __nanosleep(nap);
                        if (nap < 256) nap <<= 1;
                        if (gtime() - idle0 > wait_limit(a)) {
                            if (lane == 0) atomicCAS((int *)&S.err, 0, AOP_ETIMEOUT);
                            break;
                        }
                        continue;
                    }
                    const uint64_t tb = gtime();
                    __threadfence_block();
                    const Task t = *(const Task *)&S.tasks[pick];
                    const int lgN = c.template conv<fft::WarpGroup, StoreCell<MODE>>(
                        t.in, t.x_lo, t.x_hi, t.out, t.g, tile, a.lg_tile, wid < Shape<MODE>::big ? c.scratch(wid) : nullptr,
                        cnt);
                    __threadfence_block();
                    __syncwarp();
                    if (lane == 0) S.tasks[pick].state = TASK_DONE;
                    idle0 = gtime();
                    nap = 32;
                    if (lane == 0) {
                        cnt.busy_ns += (long long)(idle0 - tb);
                        cnt.hist_n[min(lgN, 23)]++;
                        cnt.hist_ns[min(lgN, 23)] += (long long)(idle0 - tb);
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const int err = S.err;
                a.prices[o] = err ? __longlong_as_double(0x7ff8000000000000ll) : S.price;
                if (a.greeks && (err || S.P.T < 3))
                    for (int g = 0; g < 3; g++) a.greeks[3 * o + g] = __longlong_as_double(0x7ff8000000000000ll);
                if (err) {
                    if (a.status) a.status[o] = err;
                    if (a.err) atomicCAS(a.err, 0, err);
                }
                if (a.opt_ns) {
                    uint64_t t_end;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                    a.opt_ns[o] = (int64_t)(t_end - t_start);
                }
                if (a.sreq) {
                    a.status[o] = err ? err : AOP_OK;
                    __threadfence_system();
                    a.sdone[o] = 1;
                }
            }
            __syncthreads();
        }
    }
    if (lane == 0 && a.stats) {
        atomicAdd((unsigned long long *)&a.stats->convolutions, (unsigned long long)cnt.convs);
        atomicAdd((unsigned long long *)&a.stats->fft_points, (unsigned long long)cnt.fft_points);
        atomicAdd((unsigned long long *)&a.stats->fft_flops, (unsigned long long)cnt.fft_flops);
        atomicAdd((unsigned long long *)&a.stats->conv_inputs, (unsigned long long)cnt.conv_in);
        atomicAdd((unsigned long long *)&a.stats->conv_outputs, (unsigned long long)cnt.conv_out);
        atomicAdd((unsigned long long *)&a.stats->global_fft_bytes, (unsigned long long)cnt.gbytes);
        atomicAdd((unsigned long long *)&a.stats->basecase_cells, (unsigned long long)cnt.base_cells);
        atomicAdd((unsigned long long *)&a.stats->walker_wait_ns, (unsigned long long)cnt.wait_ns);
        atomicAdd((unsigned long long *)&a.stats->worker_busy_ns, (unsigned long long)cnt.busy_ns);
        atomicAdd((unsigned long long *)&a.stats->walker_base_ns, (unsigned long long)cnt.base_ns);
        atomicAdd((unsigned long long *)&a.stats->basecase_calls, (unsigned long long)cnt.base_calls);
        atomicAdd((unsigned long long *)&a.stats->basecase_rows, (unsigned long long)cnt.base_rows);
        atomicAdd((unsigned long long *)&a.stats->walker_ns, (unsigned long long)cnt.walker_ns);
        atomicAdd((unsigned long long *)&a.stats->spectrum_ns, (unsigned long long)(cnt.spec_ns + c.cnt_spec_ns));
        atomicAdd((unsigned long long *)&a.stats->spectrum_bins, (unsigned long long)(cnt.spec_bins + c.cnt_spec_bins));
        atomicAdd((unsigned long long *)&a.stats->basecase_loop_cycles, (unsigned long long)cnt.loop_cyc);
        atomicAdd((unsigned long long *)&a.stats->basecase_fill_cycles, (unsigned long long)cnt.fill_cyc);
        for (int j = 0; j < 5; j++)
            if (cnt.cv_cyc[j]) atomicAdd((unsigned long long *)&a.stats->advance_phase_cycles[j], (unsigned long long)cnt.cv_cyc[j]);
        if (cnt.helped) {
            atomicAdd((unsigned long long *)&a.stats->helped_advances, (unsigned long long)cnt.helped);
            atomicAdd((unsigned long long *)&a.stats->helped_ns, (unsigned long long)cnt.helped_ns);
        }
        for (int j = 0; j < 24; j++) {
            if (cnt.hist_n[j]) {
                atomicAdd((unsigned long long *)&a.stats->advance_count_by_log2n[j], (unsigned long long)cnt.hist_n[j]);
                atomicAdd((unsigned long long *)&a.stats->advance_ns_by_log2n[j], (unsigned long long)cnt.hist_ns[j]);
            }
        }
    }
}

}  // namespace

}  // namespace aop
