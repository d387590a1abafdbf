// dnc.cu -- host side of the divide-and-conquer pricer: workspace layout,
// occupancy, launches, the linear-advance entry points, and the plain
// kernels (no helping; the helping ones are in dnc_help.cu).
#include "dnc_kernel.cuh"

namespace aop {

namespace {

// ------------------------------------------------------------ layout/launch
struct Layout {
    int64_t W_max, N_max, spec_cap;
    int64_t off_r0, off_mid, off_scr, off_spec, off_board, scr_stride, stride;
    int64_t mid_off[kMaxDepth];
    int lg_tile, lg_block, tw_log2, vsz;
    size_t smem;
};

int value_bytes(int method) {
    return method == AOP_FFT_FP32SPLIT ? 8 : 16;
}

Layout make_layout(int method, int64_t T_max, int B, int scratch_units, int lg_tile) {
    Layout L;
    L.vsz = value_bytes(method);
    L.W_max = 2 * T_max + 1;
    L.N_max = (int64_t)1 << ilog2_ceil(L.W_max);
    L.lg_tile = lg_tile;                      // 2^10: 8 KiB (FP32 split) or 16 KiB per worker tile
    L.lg_block = (L.vsz == 8) ? 12 : 11;     // 32 KiB block tile (linear advance entry points)
    L.tw_log2 = std::max(ilog2_ceil(L.N_max), L.lg_block + 1);
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
    L.scr_stride = (L.N_max * L.vsz + 255) & ~255ll;
    off += L.scr_stride * scratch_units;
    L.off_spec = off;
    off += (L.spec_cap * 16 + 255) & ~255ll;
    L.off_board = off;
    off += ((int64_t)sizeof(Board) + 255) & ~255ll;
    L.stride = off;
    L.smem = kNaiveCap * sizeof(double) + (size_t)shape_workers(method) * ((size_t)L.vsz << L.lg_tile);
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

template <int MODE>
int resident_ctas(size_t smem) {
    int per_sm = 0;
    cudaFuncSetAttribute(dnc_kernel<MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dnc_kernel<MODE, false>, Shape<MODE>::threads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        per_sm = 2;
    }
    return std::max(1, per_sm);
}

int ctas_per_sm(int method, size_t smem) {
    switch (method) {
    case AOP_FFT_FP64: return resident_ctas<0>(smem);
    case AOP_FFT_FP32SPLIT: return resident_ctas<1>(smem);
    default: return resident_ctas<2>(smem);
    }
}

// Dynamic shared memory that lets at most `want` CTAs share an SM, so that a
// grid of SMs x want CTAs spreads evenly (the block scheduler may otherwise
// fill some SMs up to the occupancy limit and leave others idle).
template <int MODE>
size_t spread_smem(size_t smem, int want, int device) {
    if (resident_ctas<MODE>(smem) <= want) return smem;
    int sm_bytes = 0, reserved = 0, optin = 0;
    cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, dnc_kernel<MODE, false>) != cudaSuccess) {
        cudaGetLastError();
        return smem;
    }
    size_t dyn = (size_t)(sm_bytes / want) - (size_t)reserved - fa.sharedSizeBytes;
    dyn = std::min(dyn, (size_t)optin - fa.sharedSizeBytes) & ~(size_t)127;
    while (dyn > smem && resident_ctas<MODE>(dyn) > want) dyn += 1024;     // rounding margin
    while (dyn > smem && resident_ctas<MODE>(dyn) < want) dyn -= 1024;
    dyn = std::max(dyn, smem);
    cudaFuncSetAttribute(dnc_kernel<MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    return dyn;
}

size_t spread_smem_any(int method, size_t smem, int want, int device) {
    switch (method) {
    case AOP_FFT_FP64: return spread_smem<0>(smem, want, device);
    case AOP_FFT_FP32SPLIT: return spread_smem<1>(smem, want, device);
    default: return spread_smem<2>(smem, want, device);
    }
}

}  // namespace

// Options in flight per SM: as many as fit, at most `cap`, and no more than
// needed to give every SM its share of n options.
int dnc_per_sm(int method, int64_t n, size_t smem, int cap, int device) {
    int per_sm = ctas_per_sm(method, smem);
    if (cap > 0 && cap < per_sm) per_sm = cap;
    const int64_t sms = sm_count(device);
    const int64_t share = (n + sms - 1) / sms;
    if (share >= 1 && share < per_sm) per_sm = (int)share;
    return std::max(1, per_sm);
}

// Options in flight per SM that the pricing kernel's registers and shared
// memory allow (the autotuner tries no more).
int dnc_max_per_sm(int method, int64_t T_max, int base_case, int lg_tile) {
    Layout L = make_layout(method, T_max, base_case, shape_big(method), lg_tile);
    return ctas_per_sm(method, L.smem);
}

// Helping CTAs per option of a batch of n: as many (up to kHelpers) as the
// SMs the options leave idle hold, one CTA an SM.  A helper sharing an SM
// with an option's walker slows that walker more than it saves (measured:
// 152 options of the book at T = 2^17, one owner and one helper an SM, 96-103
// against 91 ms), so batches of more than half as many options as SMs get none.
int dnc_helpers(int64_t n, int device) {
    const int64_t sms = sm_count(device);
    if (n < 1 || n >= sms) return 0;
    return (int)std::min<int64_t>(kHelpers, (sms - n) / n);
}

// One CTA per option in flight, at most n; with helping, dnc_helpers(n) more
// CTAs per option, which work for the options' boards from the start.
int64_t dnc_grid(int method, int64_t n, size_t smem, int cap, int device, bool help) {
    const int64_t m = help ? n * (1 + dnc_helpers(n, device)) : n;
    return std::min<int64_t>(m, (int64_t)sm_count(device) * dnc_per_sm(method, m, smem, cap, device));
}

size_t dnc_slot_bytes(int method, int64_t T_max, int base_case)
{
    return (size_t)make_layout(method, T_max, base_case, shape_big(method), kDefaultLgTile).stride;   // independent of the tile
}

size_t dnc_workspace_bytes(int method, int64_t n, int64_t T_max, int base_case, int cap, int *grid_out, int device,
                           int lg_tile, bool help)
{
    Layout L = make_layout(method, T_max, base_case, shape_big(method), lg_tile);
    int64_t grid = dnc_grid(method, n, L.smem, cap, device, help);
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    return (size_t)(grid * L.stride + 8192);
}

cudaError_t run_dnc(int method, int64_t n, const Params *d_params, int64_t T_max, int base_case,
                    void *ws, size_t ws_bytes, const void *d_tw, int tw_log2, double *d_prices,
                    int32_t *d_status, int32_t *d_bnd, const int64_t *d_bnd_off,
                    aop_stats *d_stats, int *d_err, int64_t *d_opt_ns, int flags, int cap, int device,
                    cudaStream_t s, const ServeSession *srv, const int32_t *d_order, double *d_greeks,
                    int lg_tile, int radix2, int base_case_put)
{
    if (srv) n = srv->capacity;
    if (n == 0) return cudaSuccess;
    if (lg_tile < 9 || lg_tile > 11) return cudaErrorInvalidValue;
    Layout L = make_layout(method, T_max, std::max(base_case, base_case_put), shape_big(method), lg_tile);
    if (tw_log2 < L.tw_log2) return cudaErrorInvalidValue;
    const bool help = !srv && !(flags & AOP_FLAG_NO_HELP) && method != AOP_FFT_FP32SPLIT &&
                      dnc_helpers(n, device) > 0;
    int64_t grid = dnc_grid(method, n, L.smem, cap, device, help);
    const size_t need = (size_t)(grid * L.stride) + 8192;
    if (ws_bytes < need) {
        grid = (int64_t)((ws_bytes - 8192) / L.stride);
        if (grid < 1) return cudaErrorMemoryAllocation;
    }
    char *base = (char *)ws;
    int *queue = (int *)(base + grid * L.stride);
    int *sm_slots = queue + 1;              // 1024 ints
    int *finished = queue + 1040;
    cudaMemsetAsync(queue, 0, 8192, s);
    DncArgs a;
    memset(&a, 0, sizeof(a));
    a.params = d_params;
    a.n = n;
    a.B = base_case;
    a.Bput = base_case_put > 0 ? base_case_put : base_case;
    a.lg_tile = L.lg_tile;
    a.radix2 = radix2 ? 1 : 0;
    a.lg_block = L.lg_block;
    a.W_max = L.W_max;
    a.ws = base;
    a.ws_stride = L.stride;
    a.off_r0 = L.off_r0;
    a.off_mid = L.off_mid;
    a.off_scr = L.off_scr;
    a.off_spec = L.off_spec;
    a.scr_stride = L.scr_stride;
    for (int d = 0; d < kMaxDepth; d++) a.mid_off[d] = L.mid_off[d];
    a.spec_cap = L.spec_cap;
    a.tw = d_tw;
    a.tw_log2 = tw_log2;
    a.prices = d_prices;
    a.status = d_status;
    a.bnd = d_bnd;
    a.bnd_off = d_bnd_off;
    a.queue = queue;
    a.sm_slots = sm_slots;
    a.grid = grid;
    a.help_lg = help ? L.lg_tile + 2 : 0;       // the multi-pass advances
    a.help_block = help && grid > n;            // CTAs launched only to help
    a.off_board = L.off_board;
    a.finished = finished;
    static std::atomic<unsigned> s_epoch{0};
    a.epoch = (s_epoch.fetch_add(1) + 1) & 0xffffffffu;
    a.err = d_err;
    a.stats = d_stats;
    a.opt_ns = d_opt_ns;
    a.greeks = srv ? nullptr : d_greeks;
    a.flags = flags;
    a.order = d_order;
    if (srv) {
        a.sreq = srv->reqs;
        a.spub = srv->pub;
        a.sstop = srv->stop;
        a.sclaim = srv->claim;
        a.sdone = srv->done;
        a.sT_max = T_max;
        a.prices = srv->prices;
        a.status = srv->status;
        a.params = nullptr;
    }
    // spread the grid: at most grid / SMs (rounded up) CTAs on any SM
    const int64_t sms = sm_count(device);
    const size_t smem = spread_smem_any(method, L.smem, (int)((grid + sms - 1) / sms), device);
    if (help) return launch_dnc_help(method, (unsigned)grid, Shape<2>::threads, smem, s, a);
    switch (method) {
    case AOP_FFT_FP64:
        dnc_kernel<0, false><<<(unsigned)grid, Shape<0>::threads, smem, s>>>(a);
        break;
    case AOP_FFT_FP32SPLIT:
        dnc_kernel<1, false><<<(unsigned)grid, Shape<1>::threads, smem, s>>>(a);
        break;
    default:
        dnc_kernel<2, false><<<(unsigned)grid, Shape<2>::threads, smem, s>>>(a);
        break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------- standalone linear advance
namespace {

template <int MODE>
__global__ void __launch_bounds__(kThreadsA) advance_kernel(const __grid_constant__ DncArgs a,
                                                            const __grid_constant__ Params P0, int64_t count,
                                                            int64_t W, int64_t h, const double *in, double *out)
{
    using V = typename fft::Cx<MODE>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared S;
    V *tile = (V *)smem_raw;
    char *slot = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    Cta<MODE> c(a, S, slot);
    Counters cnt{};
    if (threadIdx.x == 0) {
        S.P = P0;
        S.spec_n = 0;
        S.spec_lock = 0;
        for (int j = 0; j < kSpecLg * kSpecLg; j++) (&S.spec_map[0][0])[j] = 0;
        S.arena_used = 0;
        S.err = 0;
    }
    __syncthreads();
    const int64_t nout = W - (int64_t)(P0.nw - 1) * h;
    int64_t s = blockIdx.x;
    for (; s < count; s += gridDim.x) {
        Buf bi{const_cast<double *>(in) + s * W, 0};
        Buf bo{out + s * nout, 0};
        c.template conv<fft::BlockGroup, StoreF64<MODE>>(bi, 0, W - 1, bo, h, tile, a.lg_block, c.scratch(0), cnt);
        __syncthreads();
        if (S.err) break;
    }
    // A bounded wait gave up (AOP_ETIMEOUT): this segment and the block's
    // remaining ones become NaN, and the status goes to the caller's error
    // word when there is one.
    if (S.err) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        for (; s < count; s += gridDim.x)
            for (int64_t j = threadIdx.x; j < nout; j += blockDim.x) out[s * nout + j] = nan;
        if (a.err && threadIdx.x == 0) atomicCAS(a.err, 0, S.err);
    }
}

// European counterpart of an option (no early exercise): the root value is
// one T-step linear advance of the expiry payoff -- the T-fold power of the
// stencil applied to the payoff row, evaluated at the root cell -- done as one
// tilted FFT convolution by the whole CTA.  One CTA per option.
template <int MODE>
__global__ void __launch_bounds__(kThreadsA) european_kernel(const __grid_constant__ DncArgs a, double *prices,
                                                             int32_t *status)
{
    using V = typename fft::Cx<MODE>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared S;
    V *tile = (V *)smem_raw;
    char *slot = a.ws + (int64_t)blockIdx.x * a.ws_stride;
    Cta<MODE> c(a, S, slot);
    Counters cnt{};
    for (int64_t o = blockIdx.x; o < a.n; o += gridDim.x) {
        if (threadIdx.x == 0) {
            S.P = a.params[o];
            S.spec_n = 0;
            S.spec_lock = 0;
            for (int j = 0; j < kSpecLg * kSpecLg; j++) (&S.spec_map[0][0])[j] = 0;
            S.arena_used = 0;
            S.err = 0;
        }
        __syncthreads();
        if (S.P.status != AOP_OK) {
            if (threadIdx.x == 0) prices[o] = __longlong_as_double(0x7ff8000000000000ll);
            __syncthreads();
            continue;
        }
        const Params &P = S.P;
        build_exp_tables(P, S.E);
        const bool put = (P.model == AOP_BSM_PUT);
        c.tilt = !put && P.kappa > 0.0;
        if (c.tilt) build_tilt_tables<MODE>(S);
        __syncthreads();
        // expiry row: calls row T (columns 0 .. D T), the put's row 0 (k = -T .. T)
        const int64_t T = P.T;
        const int64_t W = put ? 2 * T + 1 : (int64_t)P.D * T + 1;
        double *row = (double *)(slot + a.off_r0);
        for (int64_t x = threadIdx.x; x < W; x += blockDim.x) {
            const double e = put ? exercise(P, S.E, ex_index(P, 0, x - T)) : exercise(P, S.E, ex_index(P, T, x));
            row[x] = e > 0.0 ? e : 0.0;
        }
        __syncthreads();
        double *res = (double *)(slot + a.off_mid);
        // the root: out[y] with y = x_lo - o_min T = T (put, row indexed from -T) or 0 (calls)
        const Buf bi{row, 0};
        const Buf bo{res, put ? T : 0};
        c.template conv<fft::BlockGroup, StoreF64<MODE>>(bi, 0, W - 1, bo, T, tile, a.lg_block, c.scratch(0), cnt);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int err = S.err;
            prices[o] = err ? __longlong_as_double(0x7ff8000000000000ll) : P.out_scale * res[0];
            if (status) status[o] = err ? err : AOP_OK;
        }
        __syncthreads();
    }
}

template <int MODE>
void launch_advance(const DncArgs &a, const Params &P, int64_t grid, size_t smem, int64_t count, int64_t W,
                    int64_t h, const double *d_in, double *d_out, cudaStream_t s) {
    cudaFuncSetAttribute(advance_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    advance_kernel<MODE><<<(unsigned)grid, kThreadsA, smem, s>>>(a, P, count, W, h, d_in, d_out);
}

void launch_advance_any(int method, const DncArgs &a, const Params &P, int64_t grid, size_t smem, int64_t count,
                        int64_t W, int64_t h, const double *d_in, double *d_out, cudaStream_t s) {
    if (method == AOP_FFT_FP64) launch_advance<0>(a, P, grid, smem, count, W, h, d_in, d_out, s);
    else if (method == AOP_FFT_FP32SPLIT) launch_advance<1>(a, P, grid, smem, count, W, h, d_in, d_out, s);
    else launch_advance<2>(a, P, grid, smem, count, W, h, d_in, d_out, s);
}

Params advance_params(int nw, const double *w) {
    Params P;
    memset(&P, 0, sizeof(P));
    P.model = AOP_BINOMIAL_CALL;
    P.nw = nw;
    P.D = nw - 1;
    P.o_min = 0;
    P.w[0] = w[0]; P.w[1] = w[1]; P.w[2] = nw == 3 ? w[2] : 0.0;
    P.wsum = P.w[0] + P.w[1] + P.w[2];
    for (int j = 0; j < 3; j++) P.wt[j] = P.w[j];
    P.wtsum = P.wsum;
    P.tL = 0.0;
    return P;
}

}  // namespace

size_t linear_advance_workspace_bytes(int method, int64_t W, int64_t h)
{
    (void)h;
    Layout L = make_layout(method, (W + 1) / 2 + 1, 16, 1, kDefaultLgTile);
    return (size_t)(L.stride * 64 + 4096);
}

cudaError_t run_linear_advance(int method, int nw, const double *w, int64_t count, int64_t W, int64_t h,
                               const double *d_in, double *d_out, const void *d_tw, int tw_log2,
                               void *ws, size_t ws_bytes, int *d_err, cudaStream_t s)
{
    Layout L = make_layout(method, (W + 1) / 2 + 1, 16, 1, kDefaultLgTile);
    int64_t grid = std::min<int64_t>(count, 64);
    if ((size_t)(grid * L.stride) > ws_bytes) grid = (int64_t)(ws_bytes / L.stride);
    if (grid < 1) return cudaErrorMemoryAllocation;
    if (tw_log2 < L.tw_log2) return cudaErrorInvalidValue;
    Params P = advance_params(nw, w);
    DncArgs a;
    memset(&a, 0, sizeof(a));
    a.B = 16;
    a.Bput = 16;
    a.lg_tile = L.lg_tile;
    a.lg_block = L.lg_block;
    a.W_max = L.W_max;
    a.ws = (char *)ws;
    a.ws_stride = L.stride;
    a.off_r0 = L.off_r0; a.off_mid = L.off_mid; a.off_scr = L.off_scr; a.off_spec = L.off_spec;
    a.scr_stride = L.scr_stride;
    a.spec_cap = L.spec_cap;
    a.tw = d_tw;
    a.tw_log2 = tw_log2;
    a.err = d_err;
    const size_t smem = (size_t)L.vsz << L.lg_block;
    launch_advance_any(method, a, P, grid, smem, count, W, h, d_in, d_out, s);
    return cudaGetLastError();
}

size_t european_workspace_bytes(int64_t n, int64_t T_max, int *grid_out, int device)
{
    Layout L = make_layout(AOP_FFT_FP64, T_max, 16, 1, kDefaultLgTile);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)sm_count(device) * 2));
    if (grid_out) *grid_out = (int)grid;
    return (size_t)(grid * L.stride);
}

cudaError_t run_european(int64_t n, const Params *d_params, int64_t T_max, void *ws, size_t ws_bytes,
                         const void *d_tw, int tw_log2, double *d_prices, int32_t *d_status, int device,
                         cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    Layout L = make_layout(AOP_FFT_FP64, T_max, 16, 1, kDefaultLgTile);
    if (tw_log2 < L.tw_log2) return cudaErrorInvalidValue;
    int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)sm_count(device) * 2));
    if ((size_t)(grid * L.stride) > ws_bytes) grid = (int64_t)(ws_bytes / L.stride);
    if (grid < 1) return cudaErrorMemoryAllocation;
    DncArgs a;
    memset(&a, 0, sizeof(a));
    a.params = d_params;
    a.n = n;
    a.B = 16;
    a.Bput = 16;
    a.lg_tile = L.lg_tile;
    a.lg_block = L.lg_block;
    a.W_max = L.W_max;
    a.ws = (char *)ws;
    a.ws_stride = L.stride;
    a.off_r0 = L.off_r0; a.off_mid = L.off_mid; a.off_scr = L.off_scr; a.off_spec = L.off_spec;
    a.scr_stride = L.scr_stride;
    for (int d = 0; d < kMaxDepth; d++) a.mid_off[d] = L.mid_off[d];
    a.spec_cap = L.spec_cap;
    a.tw = d_tw;
    a.tw_log2 = tw_log2;
    const size_t smem = (size_t)L.vsz << L.lg_block;
    cudaFuncSetAttribute(european_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    european_kernel<0><<<(unsigned)grid, kThreadsA, smem, s>>>(a, d_prices, d_status);
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
constexpr int64_t kNoAllocStride = kNoAllocNmax * 16 + kNoAllocSpec * 16;   // 16-byte values, worst case
constexpr int64_t kNoAllocTwEntries = (int64_t)1 << kNoAllocTwLog2;   // levels 1 .. 15
constexpr int64_t kNoAllocTw32Off = kNoAllocCtas * kNoAllocStride;
constexpr int64_t kNoAllocTw64Off = kNoAllocTw32Off + kNoAllocTwEntries * 16;
constexpr int64_t kNoAllocBytes = kNoAllocTw64Off + kNoAllocTwEntries * 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// device address of the array, looked up once per CUDA context on each device
// (host code may not use the array's name as a device pointer).  A reset
// device comes back with a new context whose copy of the array is zeroed and
// may sit elsewhere: the context's id, unique for the life of the process,
// tells the set-up to run again.
struct NoAllocDevice {
    bool ready;
    unsigned long long ctx_id;
    char *base;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// id of the calling thread's current context through the driver's entry
// points (the library links the runtime only); false if unavailable
bool current_ctx_id(unsigned long long *id) {
    typedef CUresult (*GetCurrent)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return false;
        }
        get_current = (GetCurrent)f1;
        get_id = (GetId)f2;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

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
        // the array's address in the current context (this also binds the
        // runtime's context to the thread), then that context's id
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) { cudaGetLastError(); return AOP_ECUDA; }
        unsigned long long ctx_id = 0;
        if (!current_ctx_id(&ctx_id)) return AOP_ECUDA;
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        NoAllocDevice &D = g_noalloc_dev[dev];
        if (!D.ready || D.ctx_id != ctx_id || D.base != (char *)ptr) {
            // set-up once per context on this device: fill the twiddle tables
            // the array holds (nothing is allocated)
            D.ready = false;
            char *b = (char *)ptr;
            e = launch_twiddles(kNoAllocTwLog2, b + kNoAllocTw32Off, b + kNoAllocTw64Off, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { cudaGetLastError(); return AOP_ECUDA; }
            D.base = b;
            D.ctx_id = ctx_id;
            D.ready = true;
        }
        base = D.base;
    }
    Params P = advance_params(nw, w);
    DncArgs a;
    memset(&a, 0, sizeof(a));
    a.B = 16;
    a.Bput = 16;
    a.lg_block = (method == AOP_FFT_FP64) ? 11 : 12;
    a.lg_tile = a.lg_block;
    a.W_max = kNoAllocMaxW;
    a.ws = base;
    a.ws_stride = kNoAllocStride;
    a.off_scr = 0;
    a.scr_stride = kNoAllocNmax * 16;
    a.off_spec = kNoAllocNmax * 16;
    a.spec_cap = kNoAllocSpec;
    a.tw = base + ((method == AOP_FFT_FP64) ? kNoAllocTw64Off : kNoAllocTw32Off);
    a.tw_log2 = kNoAllocTwLog2;
    a.err = nullptr;
    const int64_t grid = std::min<int64_t>(count, kNoAllocCtas);
    const size_t smem = (size_t)((method == AOP_FFT_FP64) ? 16 : 8) << a.lg_block;
    launch_advance_any(method, a, P, grid, smem, count, W, h, d_in, d_out, s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AOP_OK : AOP_ECUDA;
}
