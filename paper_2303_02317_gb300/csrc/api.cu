// api.cu -- the C ABI (include/american.h): contexts, workspace, batches.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace aop;

struct aop_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t cap = 0;
    // workspace (grow-only)
    void *ws = nullptr;
    size_t ws_size = 0;
    // per-batch device arrays (grow-only)
    void *small = nullptr;
    size_t small_size = 0;
    // pinned host staging
    void *pinned = nullptr;
    size_t pinned_size = 0;
    // twiddle tables
    void *tw32 = nullptr, *tw64 = nullptr;
    int tw_log2 = 0;
    aop_stats *d_stats = nullptr;
    int *d_err = nullptr;
    int64_t *d_tmax = nullptr;
    int64_t *d_opt_ns = nullptr;     // per-option device time of the last D&C batch
    size_t opt_ns_cap = 0;
    bool opt_ns_valid = false;
    int64_t last_n = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // bracket the pricing kernels
    bool timed = false;
    // autotuned D&C schedules, keyed by (method, log2 of the batch's largest
    // T, model class): fields 0 = not tuned
    std::map<int, aop_options> tuned;
    bool serving = false;            // a serving session holds the workspace
};

struct aop_server {
    aop_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;   // the persistent pricing kernel's stream
    int method = 0, B = 0, cap = 0, flags = 0, slots = 0, lg_tile = 0, radix2 = 0, Bput = 0;
    int64_t T_max = 0, capacity = 0;
    // host memory mapped into the device: requests in, results out
    aop_request *h_reqs = nullptr;
    double *h_prices = nullptr;
    int32_t *h_status = nullptr;
    int32_t *h_done = nullptr;
    long long *h_pub = nullptr;      // h_pub[0] = published, h_pub[1] = stop
    unsigned long long *d_claim = nullptr;
    aop_stats *d_stats = nullptr;
    int *d_err = nullptr;
    int64_t published = 0;
    int64_t first_undone = 0;        // every request below is done
    ServeSession sess{};
};

namespace {

constexpr int kDefaultBaseCase = 63;    // the tuner's usual pick: strips fill whole registers

// A D&C schedule: base-case height, options in flight per SM (0 = as many
// as fit), log2 of a worker's transform tile, radix-2-only transform stages.
struct Sched {
    int B, cap, lg_tile, radix2;
    int Bput;          // base-case height of BSM puts (their windows are four heights wide)
};
constexpr int kDefaultPutBaseCase = 31;   // a put strip of 4B + 1 cells fills four registers
// Untuned height of a batch of three-point lattices only, when the batch is
// small enough to be helped: the spare SMs absorb the extra advances of the
// lower height, and the shorter rows shorten each option's chain (measured,
// one trinomial call at T = 2^17: 54.8 ms against 63.3 at height 63; one
// binomial call stays fastest at 63).
constexpr int kHelpedTriBaseCase = 31;

aop_status cuda_fail(cudaError_t e) {
    return e == cudaSuccess ? AOP_OK : (e == cudaErrorMemoryAllocation ? AOP_ENOMEM : AOP_ECUDA);
}

#define CK(x)                                     \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

aop_status ensure(void **p, size_t *have, size_t need, size_t cap) {
    if (*have >= need) return AOP_OK;
    if (cap && need > cap) return AOP_ENOMEM;
    if (*p) { cudaFree(*p); *p = nullptr; *have = 0; }
    size_t sz = need + need / 8;
    if (cap && sz > cap) sz = need;
    cudaError_t e = cudaMalloc(p, sz);
    if (e != cudaSuccess) { cudaGetLastError(); *p = nullptr; return AOP_ENOMEM; }
    *have = sz;
    return AOP_OK;
}

aop_status ensure_pinned(aop_ctx *c, size_t need) {
    if (c->pinned_size >= need) return AOP_OK;
    if (c->pinned) cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    c->pinned_size = 0;
    size_t sz = need + need / 4 + 4096;
    if (cudaMallocHost(&c->pinned, sz) != cudaSuccess) { cudaGetLastError(); return AOP_ENOMEM; }
    c->pinned_size = sz;
    return AOP_OK;
}

aop_status ensure_twiddles(aop_ctx *c, int log2n) {
    if (c->tw_log2 >= log2n) return AOP_OK;
    if (c->tw32) cudaFree(c->tw32);
    if (c->tw64) cudaFree(c->tw64);
    c->tw32 = c->tw64 = nullptr;
    c->tw_log2 = 0;
    size_t half = (size_t)1 << (log2n - 1);
    CK(cudaMalloc(&c->tw32, 2 * half * sizeof(float4)));     // levels 1 .. log2n
    CK(cudaMalloc(&c->tw64, 2 * half * sizeof(double2)));
    CK(launch_twiddles(log2n, c->tw32, c->tw64, c->stream));
    c->tw_log2 = log2n;
    return AOP_OK;
}

// Model class of a batch for the schedule table: 0 = every option on the
// binomial lattice (two-point stencil), 1 = every option three-point
// (trinomial lattice, BSM grid), 2 = both, 3 = not known.
int model_class(int64_t n, const aop_request *reqs) {
    if (!reqs || n <= 0) return 3;
    bool two = false, three = false;
    for (int64_t i = 0; i < n; i++) {
        const int m = reqs[i].model;
        if (m == AOP_BINOMIAL_CALL || m == AOP_BINOMIAL_PUT) two = true;
        else three = true;
    }
    return (two && three) ? 2 : (two ? 0 : 1);
}

int sched_key(int method, int64_t T_max, int cls) {
    return (method * 32 + ilog2_ceil(std::max<int64_t>(T_max, 1))) * 4 + cls;
}

// The tuned schedule closest to (method, T_max, cls): the same key, else the
// same size bucket of another class, else the nearest size bucket.
aop_options lookup_tuned(const aop_ctx *c, int method, int64_t T_max, int cls) {
    aop_options none{method, 0, 0, 0, 0, 0};
    if (!c || c->tuned.empty()) return none;
    auto it = c->tuned.find(sched_key(method, T_max, cls));
    if (it != c->tuned.end()) return it->second;
    for (int k : {2, 0, 1, 3}) {
        it = c->tuned.find(sched_key(method, T_max, k));
        if (it != c->tuned.end()) return it->second;
    }
    const int lg = ilog2_ceil(std::max<int64_t>(T_max, 1));
    int best_d = 1 << 30;
    aop_options best = none;
    for (const auto &kv : c->tuned) {
        if (kv.first / 128 != method) continue;
        const int d = std::abs((kv.first / 4) % 32 - lg);
        if (d < best_d) { best_d = d; best = kv.second; }
    }
    return best;
}

// The D&C schedule of a call: explicit options first, then the context's
// tuned pick for this size and model class, then the library defaults.
Sched resolve_sched(const aop_ctx *c, const aop_options *opt, int64_t T_max, int cls, int64_t n = 0) {
    const int m = opt ? opt->method : 0;
    const aop_options t = lookup_tuned(c, m, T_max, cls);
    const bool helped = c && n > 0 && m != AOP_FFT_FP32SPLIT && !(opt && (opt->flags & AOP_FLAG_NO_HELP)) &&
                        dnc_helpers(n, c->device) > 0;
    const int B0 = (cls == 1 && helped) ? kHelpedTriBaseCase : kDefaultBaseCase;
    Sched r;
    r.B = (opt && opt->base_case > 0) ? opt->base_case : (t.base_case > 0 ? t.base_case : B0);
    r.B = std::min(64, std::max(2, r.B));
    // puts: an explicit or tuned height applies to them too; untuned, their own default
    r.Bput = (opt && opt->base_case > 0) ? r.B : (t.base_case > 0 ? r.B : kDefaultPutBaseCase);
    r.cap = (opt && opt->ctas_per_sm > 0) ? opt->ctas_per_sm : t.ctas_per_sm;
    r.lg_tile = (opt && opt->lg_tile > 0) ? opt->lg_tile : (t.lg_tile > 0 ? t.lg_tile : kDefaultLgTile);
    r.lg_tile = std::min(11, std::max(9, r.lg_tile));
    const int radix = (opt && opt->radix > 0) ? opt->radix : t.radix;
    r.radix2 = (radix == 2) ? 1 : 0;
    return r;
}

int resolve_base_case(const aop_ctx *c, const aop_options *opt) {
    return resolve_sched(c, opt, 1, 3).B;
}

// Core of every batch: d_reqs etc. on the device, T_max known.
// Longest first: the D&C grid takes options in this order, so the long ones
// start early and short ones fill the tail.  Cost estimate: T times the
// columns added per row (1 binomial, 2 trinomial and BSM).
void longest_first(int64_t n, const aop_request *reqs, int32_t *order) {
    std::vector<std::pair<int64_t, int32_t>> key((size_t)n);
    for (int64_t i = 0; i < n; i++)
        key[(size_t)i] = {-(reqs[i].T * ((reqs[i].model == AOP_BINOMIAL_CALL ||
                                          reqs[i].model == AOP_BINOMIAL_PUT) ? 1 : 2)), (int32_t)i};
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<int64_t, int32_t> &a, const std::pair<int64_t, int32_t> &b) {
                         return a.first < b.first;
                     });
    for (int64_t i = 0; i < n; i++) order[i] = key[(size_t)i].second;
}

aop_status run_batch(aop_ctx *c, int64_t n, const aop_request *d_reqs, const aop_options *opt,
                     int64_t T_max, double *d_prices, int32_t *d_status, int32_t *d_bnd,
                     const int64_t *d_bnd_off, cudaStream_t s, Params *d_params, const int32_t *d_order,
                     double *d_greeks = nullptr, int cls = 3)
{
    const int method = opt ? opt->method : AOP_FFT_FP64;
    if (method < 0 || method > 4) return AOP_EINVAL;
    const bool stencil = (method == AOP_STENCIL_FP64 || method == AOP_STENCIL_DF32);
    if (d_greeks && stencil) return AOP_EINVAL;
    if (c->serving) return AOP_EBUSY;
    if (n == 0) return AOP_OK;
    if (T_max < 1) {
        // every option was rejected (its status already says why): NaN prices
        CK(cudaMemsetAsync(d_prices, 0xff, (size_t)n * sizeof(double), s));
        return AOP_OK;
    }
    const Sched sc = resolve_sched(c, opt, T_max, cls, n);
    const int B = sc.B;
    CK(cudaMemsetAsync(c->d_stats, 0, sizeof(aop_stats), s));
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
    if (stencil) {
        size_t need = stencil_workspace_bytes(n, T_max);
        aop_status st = ensure(&c->ws, &c->ws_size, need, c->cap);
        if (st) return st;
        CK(cudaEventRecord(c->ev0, s));
        CK(run_stencil(n, d_params, T_max, c->ws, d_prices, d_status, d_bnd, d_bnd_off, c->d_stats, s,
                       method == AOP_STENCIL_DF32));
        CK(cudaEventRecord(c->ev1, s));
    } else {
        int64_t W = 2 * T_max + 1;
        int lg = ilog2_ceil(W);
        if (lg < 13) lg = 13;
        aop_status st = ensure_twiddles(c, lg);
        if (st) return st;
        int grid = 0;
        const int cap = sc.cap;
        size_t need = dnc_workspace_bytes(method, n, T_max, std::max(B, sc.Bput), cap, &grid, c->device,
                                          sc.lg_tile, !(opt && (opt->flags & AOP_FLAG_NO_HELP)) && method != AOP_FFT_FP32SPLIT);
        size_t have_cap = c->cap ? c->cap : need;
        if (need > have_cap) need = have_cap;   // fewer resident CTAs
        st = ensure(&c->ws, &c->ws_size, need, c->cap);
        if (st) return st;
        const void *tw = (method == AOP_FFT_FP64) ? c->tw64 : c->tw32;
        int64_t *opt_ns = nullptr;
        c->opt_ns_valid = false;
        if (opt && (opt->flags & AOP_FLAG_OPTION_TIMES)) {
            st = ensure((void **)&c->d_opt_ns, &c->opt_ns_cap, (size_t)n * sizeof(int64_t), 0);
            if (st) return st;
            opt_ns = c->d_opt_ns;
            c->opt_ns_valid = true;
        }
        CK(cudaEventRecord(c->ev0, s));
        CK(run_dnc(method, n, d_params, T_max, B, c->ws, c->ws_size, tw, c->tw_log2, d_prices,
                   d_status, d_bnd, d_bnd_off, c->d_stats, c->d_err, opt_ns, opt ? opt->flags : 0,
                   cap, c->device, s, nullptr, d_order, d_greeks, sc.lg_tile, sc.radix2, sc.Bput));
        CK(cudaEventRecord(c->ev1, s));
    }
    // lattice puts ran as mirrored calls: map their dividers back
    if (d_bnd) CK(launch_mirror_boundaries(n, d_params, d_bnd, d_bnd_off, s));
    c->timed = true;
    c->last_n = n;
    return AOP_OK;
}

std::mutex g_default_mu;
aop_ctx *g_default[64];

aop_ctx *default_ctx(int device, aop_status *st) {
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (device < 0 || device >= 64) { *st = AOP_EINVAL; return nullptr; }
    if (!g_default[device]) {
        aop_ctx *c = nullptr;
        *st = aop_ctx_create(&c, device, 0);
        if (*st) return nullptr;
        g_default[device] = c;
    }
    *st = AOP_OK;
    return g_default[device];
}

}  // namespace

extern "C" {

const char *aop_status_string(aop_status s) {
    switch (s) {
    case AOP_OK: return "ok";
    case AOP_EINVAL: return "invalid argument";
    case AOP_EUNSTABLE: return "negative lattice probability or finite-difference weight";
    case AOP_ENOMEM: return "workspace cap exceeded or device allocation failed";
    case AOP_ECUDA: return "CUDA runtime error or no usable device";
    case AOP_ETIMEOUT: return "bounded device wait gave up";
    case AOP_EBUSY: return "no workspace slot free";
    case AOP_EINTERNAL: return "device-side consistency check failed";
    case AOP_ERANGE: return "continuation values beyond the FP32 range (use AOP_FFT_FP64)";
    }
    return "unknown status";
}

const char *aop_version(void) { return "paper_2303_02317_gb300 0.1 (sm_103a)"; }

aop_status aop_ctx_create(aop_ctx **ctx, int device, size_t workspace_cap_bytes) {
    if (!ctx) return AOP_EINVAL;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { cudaGetLastError(); return AOP_ECUDA; }
    if (device < 0 || device >= ndev) return AOP_EINVAL;
    aop_ctx *c = new aop_ctx();
    c->device = device;
    c->cap = workspace_cap_bytes ? workspace_cap_bytes : ((size_t)64 << 30);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_stats, sizeof(aop_stats));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tmax, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, sizeof(aop_stats));
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        aop_ctx_destroy(c);
        return cuda_fail(e);
    }
    *ctx = c;
    return AOP_OK;
}

aop_status aop_ctx_destroy(aop_ctx *c) {
    if (!c) return AOP_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->small) cudaFree(c->small);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->tw32) cudaFree(c->tw32);
    if (c->tw64) cudaFree(c->tw64);
    if (c->d_stats) cudaFree(c->d_stats);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_tmax) cudaFree(c->d_tmax);
    if (c->d_opt_ns) cudaFree(c->d_opt_ns);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return AOP_OK;
}

aop_status price_american_batch_device(aop_ctx *c, int64_t n, const aop_request *d_reqs,
                                       const aop_options *opt, double *d_prices, int32_t *d_status,
                                       int32_t *d_bnd, const int64_t *d_bnd_off, void *stream) {
    if (!c || n < 0 || (n > 0 && (!d_reqs || !d_prices)) || (d_bnd && !d_bnd_off)) return AOP_EINVAL;
    if (n == 0) return AOP_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    // per-batch device arrays: params | order
    const size_t off_ord = ((size_t)n * sizeof(Params) + 255) & ~(size_t)255;
    aop_status st = ensure(&c->small, &c->small_size, off_ord + (size_t)n * sizeof(int32_t) + 256, 0);
    if (st) return st;
    Params *d_params = (Params *)c->small;
    int32_t *d_order = (int32_t *)((char *)c->small + off_ord);
    const size_t rb = (size_t)n * sizeof(aop_request);
    if ((st = ensure_pinned(c, rb + (size_t)n * sizeof(int32_t) + 64))) return st;
    aop_request *h_reqs = (aop_request *)c->pinned;
    int32_t *h_order = (int32_t *)((char *)c->pinned + rb);
    CK(cudaMemsetAsync(c->d_tmax, 0, sizeof(int64_t), s));
    CK(launch_params(n, d_reqs, d_params, d_status, c->d_tmax, s));
    int64_t T_max = 0;
    CK(cudaMemcpyAsync(&T_max, c->d_tmax, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_reqs, d_reqs, rb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (T_max == 0) {
        // every option was rejected: fill NaN prices
        CK(cudaMemsetAsync(d_prices, 0xff, (size_t)n * sizeof(double), s));
        return AOP_OK;
    }
    longest_first(n, h_reqs, h_order);
    CK(cudaMemcpyAsync(d_order, h_order, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    return run_batch(c, n, d_reqs, opt, T_max, d_prices, d_status, d_bnd, d_bnd_off, s, d_params, d_order,
                     nullptr, model_class(n, h_reqs));
}

// Host-array batch, with optional sensitivities (greeks: 3 doubles per option).
static aop_status host_batch(aop_ctx *c, int64_t n, const aop_request *reqs, const aop_options *opt,
                             double *prices, double *greeks, aop_status *status, void *stream) {
    if (!c || n < 0 || (n > 0 && (!reqs || !prices))) return AOP_EINVAL;
    if (n == 0) return AOP_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const size_t rb = (size_t)n * sizeof(aop_request), pb = (size_t)n * sizeof(double),
                 sb = (size_t)n * sizeof(int32_t);
    const size_t ob = (size_t)n * sizeof(int32_t);
    const size_t gb = greeks ? 3 * (size_t)n * sizeof(double) : 0;
    aop_status st = ensure_pinned(c, rb + pb + sb + ob + gb + 64);
    if (st) return st;
    // device arrays: reqs | prices | status | params | order | greeks
    size_t off_p = (rb + 255) & ~(size_t)255, off_s = (off_p + pb + 255) & ~(size_t)255,
           off_par = (off_s + sb + 255) & ~(size_t)255,
           off_ord = (off_par + (size_t)n * sizeof(Params) + 255) & ~(size_t)255,
           off_g = (off_ord + ob + 255) & ~(size_t)255;
    st = ensure(&c->small, &c->small_size, off_g + gb + 256, 0);
    if (st) return st;
    char *d = (char *)c->small;
    aop_request *d_reqs = (aop_request *)d;
    double *d_prices = (double *)(d + off_p);
    int32_t *d_status = (int32_t *)(d + off_s);
    Params *d_params = (Params *)(d + off_par);
    int32_t *d_order = (int32_t *)(d + off_ord);
    double *d_greeks = greeks ? (double *)(d + off_g) : nullptr;
    char *h = (char *)c->pinned;
    memcpy(h, reqs, rb);
    int32_t *h_order = (int32_t *)(h + rb + pb + sb);
    double *h_greeks = (double *)(h + rb + pb + sb + ob);
    longest_first(n, reqs, h_order);
    int64_t T_max = 0;
    for (int64_t i = 0; i < n; i++)
        if (reqs[i].T > T_max && reqs[i].T <= AOP_MAX_T) T_max = reqs[i].T;
    CK(cudaMemcpyAsync(d_reqs, h, rb, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_order, h_order, ob, cudaMemcpyHostToDevice, s));
    CK(launch_params(n, d_reqs, d_params, d_status, nullptr, s));
    if (d_greeks) CK(cudaMemsetAsync(d_greeks, 0xff, gb, s));     // NaN for rejected options
    st = run_batch(c, n, d_reqs, opt, T_max, d_prices, d_status, nullptr, nullptr, s, d_params, d_order,
                   d_greeks, model_class(n, reqs));
    if (st) return st;
    CK(cudaMemcpyAsync(h + rb, d_prices, pb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + rb + pb, d_status, sb, cudaMemcpyDeviceToHost, s));
    if (d_greeks) CK(cudaMemcpyAsync(h_greeks, d_greeks, gb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memcpy(prices, h + rb, pb);
    if (greeks) memcpy(greeks, h_greeks, gb);
    if (status) {
        const int32_t *hs = (const int32_t *)(h + rb + pb);
        for (int64_t i = 0; i < n; i++) status[i] = (aop_status)hs[i];
    }
    return AOP_OK;
}

aop_status price_american_batch(aop_ctx *c, int64_t n, const aop_request *reqs, const aop_options *opt,
                                double *prices, aop_status *status, void *stream) {
    return host_batch(c, n, reqs, opt, prices, nullptr, status, stream);
}

aop_status price_american_greeks_batch(aop_ctx *c, int64_t n, const aop_request *reqs, const aop_options *opt,
                                       double *prices, double *greeks, aop_status *status, void *stream) {
    if (n > 0 && !greeks) return AOP_EINVAL;
    return host_batch(c, n, reqs, opt, prices, greeks, status, stream);
}

aop_status price_european_batch(aop_ctx *c, int64_t n, const aop_request *reqs, double *prices,
                                aop_status *status) {
    if (!c || n < 0 || (n > 0 && (!reqs || !prices))) return AOP_EINVAL;
    if (n == 0) return AOP_OK;
    if (c->serving) return AOP_EBUSY;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const size_t rb = (size_t)n * sizeof(aop_request), pb = (size_t)n * sizeof(double),
                 sb = (size_t)n * sizeof(int32_t);
    aop_status st = ensure_pinned(c, rb + pb + sb + 64);
    if (st) return st;
    size_t off_p = (rb + 255) & ~(size_t)255, off_s = (off_p + pb + 255) & ~(size_t)255,
           off_par = (off_s + sb + 255) & ~(size_t)255;
    if ((st = ensure(&c->small, &c->small_size, off_par + (size_t)n * sizeof(Params) + 256, 0))) return st;
    char *d = (char *)c->small;
    aop_request *d_reqs = (aop_request *)d;
    double *d_prices = (double *)(d + off_p);
    int32_t *d_status = (int32_t *)(d + off_s);
    Params *d_params = (Params *)(d + off_par);
    char *h = (char *)c->pinned;
    memcpy(h, reqs, rb);
    int64_t T_max = 0;
    for (int64_t i = 0; i < n; i++)
        if (reqs[i].T > T_max && reqs[i].T <= AOP_EUROPEAN_MAX_T) T_max = reqs[i].T;
    if (T_max == 0) T_max = 1;
    int lg = ilog2_ceil(2 * T_max + 1);
    if (lg < 13) lg = 13;
    if ((st = ensure_twiddles(c, lg + 1))) return st;
    int grid = 0;
    size_t need = european_workspace_bytes(n, T_max, &grid, c->device);
    if (c->cap && need > c->cap) need = c->cap;
    if ((st = ensure(&c->ws, &c->ws_size, need, c->cap))) return st;
    CK(cudaMemcpyAsync(d_reqs, h, rb, cudaMemcpyHostToDevice, s));
    CK(launch_params(n, d_reqs, d_params, d_status, nullptr, s));
    CK(cudaEventRecord(c->ev0, s));
    CK(run_european(n, d_params, T_max, c->ws, c->ws_size, c->tw64, c->tw_log2, d_prices, d_status, c->device,
                    s));
    CK(cudaEventRecord(c->ev1, s));
    c->timed = true;
    c->last_n = n;
    CK(cudaMemcpyAsync(h + rb, d_prices, pb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + rb + pb, d_status, sb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memcpy(prices, h + rb, pb);
    const int32_t *hs = (const int32_t *)(h + rb + pb);
    for (int64_t i = 0; i < n; i++) {
        aop_status e = (aop_status)hs[i];
        if (e == AOP_OK && reqs[i].T > AOP_EUROPEAN_MAX_T) e = AOP_EINVAL;
        if (e != AOP_OK) prices[i] = __builtin_nan("");
        if (status) status[i] = e;
    }
    return AOP_OK;
}

aop_status price_american_ex(const aop_request *req, const aop_options *opt, double *price_out,
                             int32_t *boundary_out) {
    if (!req || !price_out) return AOP_EINVAL;
    if (req->T < 1 || req->T > AOP_MAX_T) return AOP_EINVAL;
    aop_status st;
    aop_ctx *c = default_ctx(0, &st);
    if (!c) return st;
    std::lock_guard<std::mutex> lk(g_default_mu);
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const int64_t T = req->T;
    // device: req | price | status | boundary | offset | params
    size_t off_price = 256, off_stat = 512, off_off = 768, off_par = 1024,
           off_b = off_par + ((sizeof(Params) + 255) & ~(size_t)255);
    size_t need = off_b + (size_t)(T + 1) * sizeof(int32_t) + 256;
    st = ensure(&c->small, &c->small_size, need, 0);
    if (st) return st;
    char *d = (char *)c->small;
    st = ensure_pinned(c, (size_t)(T + 1) * sizeof(int32_t) + 512);
    if (st) return st;
    char *h = (char *)c->pinned;
    memcpy(h, req, sizeof(aop_request));
    int64_t zero = 0;
    memcpy(h + 128, &zero, sizeof(zero));
    CK(cudaMemcpyAsync(d, h, sizeof(aop_request), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d + off_off, h + 128, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    Params *d_params = (Params *)(d + off_par);
    int32_t *d_status = (int32_t *)(d + off_stat);
    CK(launch_params(1, (const aop_request *)d, d_params, d_status, nullptr, s));
    int32_t *d_b = boundary_out ? (int32_t *)(d + off_b) : nullptr;
    st = run_batch(c, 1, (const aop_request *)d, opt, T, (double *)(d + off_price), d_status, d_b,
                   (const int64_t *)(d + off_off), s, d_params, nullptr, nullptr, model_class(1, req));
    if (st) return st;
    CK(cudaMemcpyAsync(h + 256, d + off_price, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + 264, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (d_b) CK(cudaMemcpyAsync(h + 512, d_b, (size_t)(T + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int32_t ost;
    memcpy(price_out, h + 256, sizeof(double));
    memcpy(&ost, h + 264, sizeof(int32_t));
    if (d_b) memcpy(boundary_out, h + 512, (size_t)(T + 1) * sizeof(int32_t));
    return (aop_status)ost;
}

aop_status price_american(int model, double S0, double K, double r, double q, double sigma, double expiry,
                          int64_t T, double *price_out) {
    aop_request rq;
    memset(&rq, 0, sizeof(rq));
    rq.model = model;
    rq.tri_form = AOP_TRI_BOYLE;
    rq.S0 = S0; rq.K = K; rq.r = r; rq.q = q; rq.sigma = sigma; rq.expiry = expiry;
    rq.T = T;
    rq.lambda = 0.0;
    aop_options o;
    memset(&o, 0, sizeof(o));
    o.method = AOP_FFT_FP64;
    return price_american_ex(&rq, &o, price_out, nullptr);
}

aop_status aop_linear_advance_device(aop_ctx *c, int method, int nw, const double *w, int64_t count,
                                     int64_t W, int64_t h, const double *d_in, double *d_out, void *stream) {
    if (!c || !w || !d_in || !d_out) return AOP_EINVAL;
    if (method != AOP_FFT_FP64 && method != AOP_FFT_FP32SPLIT && method != AOP_FFT_DF32) return AOP_EINVAL;
    if (nw < 2 || nw > 3 || h < 1 || count < 0 || W > ((int64_t)1 << 20) || (int64_t)(nw - 1) * h >= W)
        return AOP_EINVAL;
    if (count == 0) return AOP_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    int lg = ilog2_ceil(W + 2);
    if (lg < 13) lg = 13;
    aop_status st = ensure_twiddles(c, lg + 1);
    if (st) return st;
    size_t need = linear_advance_workspace_bytes(method, W, h);
    st = ensure(&c->ws, &c->ws_size, need, c->cap);
    if (st) return st;
    const void *tw = (method == AOP_FFT_FP64) ? c->tw64 : c->tw32;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
    CK(run_linear_advance(method, nw, w, count, W, h, d_in, d_out, tw, c->tw_log2, c->ws, c->ws_size,
                          c->d_err, s));
    int err = 0;
    CK(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return err ? (aop_status)err : AOP_OK;
}

aop_status aop_ctx_get_option_times(aop_ctx *c, int64_t n, int64_t *ns_out) {
    if (!c || !ns_out || n < 0) return AOP_EINVAL;
    if (!c->opt_ns_valid || n > c->last_n) return AOP_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(ns_out, c->d_opt_ns, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToHost));
    return AOP_OK;
}

aop_status aop_ctx_autotune(aop_ctx *c, int64_t n, const aop_request *reqs, int32_t method,
                            aop_options *best_out) {
    return aop_ctx_autotune_flags(c, n, reqs, method, 0, best_out);
}

aop_status aop_ctx_autotune_flags(aop_ctx *c, int64_t n, const aop_request *reqs, int32_t method, int32_t flags,
                                  aop_options *best_out) {
    if (!c || n <= 0 || !reqs || method < 0 || method > 3 || method == AOP_STENCIL_FP64) return AOP_EINVAL;   // D&C only
    // heights 2^k - 1 fit a binomial strip (B + 1 cells) or a trinomial one
    // (2B + 2 cells) into whole registers of 32 cells
    static const int kB[] = {16, 31, 32, 47, 63, 64};
    static const int kCap[] = {1, 2, 3, 4};
    static const int kLgTile[] = {9, 10, 11};
    static const int kRadix[] = {4, 2};
    int64_t T_max = 1;
    for (int64_t i = 0; i < n; i++) T_max = std::max<int64_t>(T_max, reqs[i].T);
    std::vector<double> prices((size_t)n);
    std::vector<aop_status> status((size_t)n);
    float best = -1.f;
    aop_options pick{method, kDefaultBaseCase, 0, 0, kDefaultLgTile, 4};
    auto time_one = [&](const aop_options &o, float *ms) -> aop_status {
        for (int rep = 0; rep < 2; rep++) {   // the first run sizes the workspace
            aop_status st = price_american_batch(c, n, reqs, &o, prices.data(), status.data(), nullptr);
            if (st) return st;
            CK(cudaEventElapsedTime(ms, c->ev0, c->ev1));
        }
        return AOP_OK;
    };
    // stage 1: base-case height x options in flight per SM x radix at the
    // default tile (height, count and radix trade walker time against worker
    // time and code size together, so they are searched jointly)
    for (int radix : kRadix) {
        for (int B : kB) {
            for (int cap : kCap) {
                if (cap > 1 && cap > dnc_max_per_sm(method, T_max, B)) continue;   // same as fewer
                aop_options o{method, B, flags, cap, kDefaultLgTile, radix};
                float ms = 0.f;
                aop_status st = time_one(o, &ms);
                if (st) return st;
                if (best < 0.f || ms < best) { best = ms; pick = o; }
            }
        }
    }
    // stage 2: the transform tile at that pick
    for (int lg : kLgTile) {
        if (lg == kDefaultLgTile) continue;                     // timed in stage 1
        if (pick.ctas_per_sm > 1 && pick.ctas_per_sm > dnc_max_per_sm(method, T_max, pick.base_case, lg))
            continue;                                           // the tile leaves no room for the count
        aop_options o{method, pick.base_case, flags, pick.ctas_per_sm, lg, pick.radix};
        float ms = 0.f;
        aop_status st = time_one(o, &ms);
        if (st) return st;
        if (ms < best) { best = ms; pick = o; }
    }
    // stage 3: when stage 2 moved the tile, the height and count again at it
    if (pick.lg_tile != kDefaultLgTile) {
        const aop_options at = pick;
        for (int B : kB) {
            for (int cap : kCap) {
                if (B == at.base_case && cap == at.ctas_per_sm) continue;
                if (cap > 1 && cap > dnc_max_per_sm(method, T_max, B, at.lg_tile)) continue;
                aop_options o{method, B, flags, cap, at.lg_tile, at.radix};
                float ms = 0.f;
                aop_status st = time_one(o, &ms);
                if (st) return st;
                if (ms < best) { best = ms; pick = o; }
            }
        }
    }
    pick.flags = 0;
    c->tuned[sched_key(method, T_max, model_class(n, reqs))] = pick;
    if (best_out) *best_out = pick;
    return AOP_OK;
}

aop_status aop_ctx_schedule(const aop_ctx *c, int64_t n, const aop_request *reqs, const aop_options *opt,
                            aop_options *out) {
    if (!c || !out || n <= 0 || !reqs || !opt) return AOP_EINVAL;
    const int method = opt->method;
    if (method < 0 || method > 3 || method == AOP_STENCIL_FP64) return AOP_EINVAL;   // D&C only
    int64_t T_max = 1;
    for (int64_t i = 0; i < n; i++) T_max = std::max<int64_t>(T_max, reqs[i].T);
    const Sched sc = resolve_sched(c, opt, T_max, model_class(n, reqs), n);
    *out = aop_options{method, sc.B, opt->flags, sc.cap, sc.lg_tile, sc.radix2 ? 2 : 4};
    return AOP_OK;
}

// ------------------------------------------------------------ serving
namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

aop_status server_launch(aop_server *s) {
    aop_ctx *c = s->ctx;
    const void *tw = (s->method == AOP_FFT_FP64) ? c->tw64 : c->tw32;
    CK(run_dnc(s->method, s->capacity, nullptr, s->T_max, s->B, c->ws, c->ws_size, tw, c->tw_log2, nullptr,
               nullptr, nullptr, nullptr, s->d_stats, s->d_err, nullptr, s->flags, s->cap, c->device, s->stream,
               &s->sess, nullptr, nullptr, s->lg_tile, s->radix2, s->Bput));
    return AOP_OK;
}

bool server_done(const aop_server *s, int64_t id) {
    return __atomic_load_n(&s->h_done[id], __ATOMIC_ACQUIRE) != 0;
}

// The persistent kernel exits after kIdleNs without a published request (and
// on stop); relaunch it while published requests are still undone.
aop_status server_ensure_running(aop_server *s) {
    while (s->first_undone < s->published && server_done(s, s->first_undone)) s->first_undone++;
    if (s->first_undone >= s->published) return AOP_OK;
    const cudaError_t q = cudaStreamQuery(s->stream);
    if (q == cudaErrorNotReady) return AOP_OK;
    if (q != cudaSuccess) return cuda_fail(q);
    if (__atomic_load_n(&s->h_pub[1], __ATOMIC_ACQUIRE)) return AOP_OK;
    return server_launch(s);
}

}  // namespace

aop_status aop_server_create(aop_ctx *c, int64_t capacity, int64_t T_max, const aop_options *opt,
                             aop_server **out) {
    if (!c || !out || capacity < 1 || T_max < 1 || T_max > AOP_MAX_T) return AOP_EINVAL;
    const int method = opt ? opt->method : AOP_FFT_FP64;
    if (method < 0 || method > 3 || method == AOP_STENCIL_FP64) return AOP_EINVAL;   // D&C only
    if (c->serving) return AOP_EBUSY;
    CK(cudaSetDevice(c->device));
    aop_server *s = new aop_server;
    s->ctx = c;
    s->method = method;
    const Sched sc = resolve_sched(c, opt, T_max, 2);
    s->B = sc.B;
    s->Bput = sc.Bput;
    s->cap = sc.cap;
    s->lg_tile = sc.lg_tile;
    s->radix2 = sc.radix2;
    s->flags = opt ? (opt->flags & ~AOP_FLAG_OPTION_TIMES) : 0;
    s->T_max = T_max;
    s->capacity = capacity;
    aop_status st = AOP_OK;
    auto fail = [&](aop_status e) {
        aop_server_destroy(s);
        return e;
    };
    int lg = ilog2_ceil(2 * T_max + 1);
    if (lg < 13) lg = 13;
    if ((st = ensure_twiddles(c, lg))) return fail(st);
    int grid = 0;
    size_t need = dnc_workspace_bytes(method, capacity, T_max, std::max(s->B, s->Bput), s->cap, &grid, c->device,
                                      s->lg_tile);
    if (c->cap && need > c->cap) need = c->cap;     // admission: the slots the cap holds
    if ((st = ensure(&c->ws, &c->ws_size, need, c->cap))) return fail(st);
    // the slots the workspace holds (the launch clips its grid the same way)
    const size_t stride = dnc_slot_bytes(method, T_max, std::max(s->B, s->Bput));
    if (c->ws_size < stride + 8192) return fail(AOP_ENOMEM);
    s->slots = (int)std::min<int64_t>(grid, (int64_t)((c->ws_size - 8192) / stride));
    const size_t per = sizeof(aop_request) + sizeof(double) + 2 * sizeof(int32_t);
    char *h = nullptr;
    if (cudaHostAlloc((void **)&h, (size_t)capacity * per + 256, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess) {
        cudaGetLastError();
        return fail(AOP_ENOMEM);
    }
    memset(h, 0, (size_t)capacity * per + 256);
    s->h_pub = (long long *)h;
    s->h_reqs = (aop_request *)(h + 64);
    s->h_prices = (double *)(s->h_reqs + capacity);
    s->h_status = (int32_t *)(s->h_prices + capacity);
    s->h_done = s->h_status + capacity;
    char *d = nullptr;
    if (cudaHostGetDevicePointer((void **)&d, h, 0) != cudaSuccess) return fail(AOP_ECUDA);
    s->sess.pub = (const volatile long long *)d;
    s->sess.stop = (const volatile int *)(d + sizeof(long long));
    s->sess.reqs = (const aop_request *)(d + 64);
    s->sess.prices = (double *)(d + 64 + capacity * sizeof(aop_request));
    s->sess.status = (int32_t *)(d + 64 + capacity * (sizeof(aop_request) + sizeof(double)));
    s->sess.done = (volatile int32_t *)(d + 64 + capacity * (sizeof(aop_request) + sizeof(double) +
                                                               sizeof(int32_t)));
    s->sess.capacity = capacity;
    if (cudaMalloc(&s->d_claim, 64) != cudaSuccess || cudaMalloc(&s->d_stats, sizeof(aop_stats)) != cudaSuccess ||
        cudaMalloc(&s->d_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(AOP_ENOMEM);
    }
    s->sess.claim = s->d_claim;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(AOP_ECUDA);
    CK(cudaMemsetAsync(s->d_claim, 0, 64, s->stream));
    CK(cudaMemsetAsync(s->d_stats, 0, sizeof(aop_stats), s->stream));
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
    c->serving = true;
    if ((st = server_launch(s))) return fail(st);
    *out = s;
    return AOP_OK;
}

aop_status aop_server_submit(aop_server *s, const aop_request *req, int64_t *id_out) {
    if (!s || !req) return AOP_EINVAL;
    if (s->published >= s->capacity) return AOP_EBUSY;
    const int64_t id = s->published;
    s->h_reqs[id] = *req;
    __atomic_store_n(&s->h_pub[0], (long long)(id + 1), __ATOMIC_RELEASE);
    s->published = id + 1;
    if (id_out) *id_out = id;
    return server_ensure_running(s);
}

aop_status aop_server_poll(aop_server *s, int64_t id, double *price, aop_status *status, int32_t *done) {
    if (!s || !done || id < 0 || id >= s->published) return AOP_EINVAL;
    *done = server_done(s, id) ? 1 : 0;
    if (*done) {
        if (price) *price = s->h_prices[id];
        if (status) *status = (aop_status)s->h_status[id];
    }
    return server_ensure_running(s);
}

aop_status aop_server_serve_stream(aop_server *s, int64_t n, const aop_request *reqs, const int64_t *arrival_ns,
                                   double *prices, aop_status *status, int64_t *latency_ns, double timeout_s) {
    if (!s || n < 0 || (n > 0 && (!reqs || !arrival_ns))) return AOP_EINVAL;
    if (s->published + n > s->capacity) return AOP_EBUSY;
    const int64_t base = s->published;
    std::vector<int64_t> pending;
    pending.reserve(4096);
    std::vector<int64_t> t_done((size_t)n, -1);
    const int64_t t0 = now_ns();
    const int64_t limit = t0 + (int64_t)(timeout_s * 1e9) + (n ? arrival_ns[n - 1] : 0);
    int64_t next = 0, left = n;
    aop_status st = AOP_OK;
    auto sweep = [&]() {
        const int64_t t = now_ns();
        size_t w = 0;
        for (size_t k = 0; k < pending.size(); k++) {
            const int64_t i = pending[k];
            if (server_done(s, base + i)) {
                t_done[(size_t)i] = t;
                left--;
            } else {
                pending[w++] = i;
            }
        }
        pending.resize(w);
    };
    while (left > 0) {
        const int64_t t = now_ns();
        while (next < n && t - t0 >= arrival_ns[next]) {
            if ((st = aop_server_submit(s, &reqs[next], nullptr))) return st;
            pending.push_back(next);
            next++;
        }
        sweep();
        if ((st = server_ensure_running(s))) return st;
        if (now_ns() > limit) return AOP_ETIMEOUT;
    }
    for (int64_t i = 0; i < n; i++) {
        if (prices) prices[i] = s->h_prices[base + i];
        if (status) status[i] = (aop_status)s->h_status[base + i];
        if (latency_ns) latency_ns[i] = t_done[(size_t)i] - (t0 + arrival_ns[i]);
    }
    return AOP_OK;
}

aop_status aop_workspace_bytes(int method, int64_t T_max, int base_case, int64_t options_in_flight,
                               size_t *bytes_out) {
    if (!bytes_out || T_max < 1 || T_max > AOP_MAX_T || options_in_flight < 1 || base_case < 0) return AOP_EINVAL;
    if (method < 0 || method > 3 || method == AOP_STENCIL_FP64) return AOP_EINVAL;   // D&C only
    aop_options o{method, base_case, 0, 0};
    const int B = resolve_base_case(nullptr, &o);
    *bytes_out = dnc_slot_bytes(method, T_max, std::max(B, kDefaultPutBaseCase)) * (size_t)options_in_flight + 8192;
    return AOP_OK;
}

aop_status aop_server_info(const aop_server *s, int64_t *slots, int64_t *published) {
    if (!s) return AOP_EINVAL;
    if (slots) *slots = s->slots;
    if (published) *published = s->published;
    return AOP_OK;
}

aop_status aop_server_destroy(aop_server *s) {
    if (!s) return AOP_EINVAL;
    if (s->h_pub) __atomic_store_n(&s->h_pub[1], 1ll, __ATOMIC_RELEASE);
    if (s->stream) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
    }
    if (s->h_pub) cudaFreeHost(s->h_pub);
    if (s->d_claim) cudaFree(s->d_claim);
    if (s->d_stats) cudaFree(s->d_stats);
    if (s->d_err) cudaFree(s->d_err);
    if (s->ctx) s->ctx->serving = false;
    delete s;
    return AOP_OK;
}

aop_status aop_ctx_get_stats(aop_ctx *c, aop_stats *out) {
    if (!c || !out) return AOP_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(out, c->d_stats, sizeof(aop_stats), cudaMemcpyDeviceToHost));
    out->options = c->last_n;
    out->kernel_ms = 0.0;
    if (c->timed) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        out->kernel_ms = ms;
    }
    return AOP_OK;
}

}  // extern "C"
