/*
 * american.h -- C ABI of the GB300 (sm_103a) nonlinear-stencil American option
 * pricer: an implementation of the trapezoidal divide-and-conquer of
 * "Fast American Option Pricing using Nonlinear Stencils" (arXiv 2303.02317),
 * plus the plain Theta(T^2) lattice loop it replaces.
 *
 * Conventions for every entry point
 *   - Status codes only; nothing throws across this boundary.
 *   - The caller owns every buffer passed in.  The library owns only the device
 *     workspace held by an aop_ctx; nothing the library allocates crosses the ABI.
 *   - Host pointers are plain C arrays.  Entry points whose names end in
 *     "_device" take device pointers (memory allocated on the context's device)
 *     and run asynchronously on the given CUDA stream (cudaStream_t passed as
 *     void*; NULL = the context's own stream).
 *   - A context is used by one host thread at a time; contexts are independent.
 *   - Every computation runs in the library's CUDA kernels.  If no CUDA device
 *     is usable the entry points return AOP_ECUDA; there is no CPU fallback.
 */
#ifndef AMERICAN_H
#define AMERICAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Lattice models.
 *   AOP_BINOMIAL_CALL  -- Sec. 2 (Fig. 1, Def. 2.1): (T+1)x(T+1) grid, row i
 *       holds columns j in [0, i] at price S0 u^{2j-i}, u = e^{sigma sqrt(dt)},
 *       dt = expiry/T; weights m(1-p) on G[i+1][j] and m p on G[i+1][j+1].
 *   AOP_TRINOMIAL_CALL -- Sec. 3 and its appendix: row i holds j in [0, 2i] at
 *       price S0 u^{j-i}; weights m p_d, m p_o, m p_u on G[i+1][j..j+2].
 *   AOP_BSM_PUT        -- Sec. 4: explicit finite differences for the
 *       nondimensional Black-Scholes-Merton put (scheme bsmG) on the shrinking
 *       triangle k in [-(T-n), T-n], dtau = sigma^2 expiry/(2T),
 *       ds = sqrt(3 dtau), s_k = ln(S0/K) + k ds.  A dividend yield q (not in
 *       the paper) sets the first-derivative coefficient to 2(r-q)/sigma^2 - 1;
 *       the discount term keeps omega = 2r/sigma^2.
 *   AOP_BINOMIAL_PUT, AOP_TRINOMIAL_PUT -- the two lattices above with the
 *       put's exercise value K - S0 u^x (Sec. 2.1 states it; the paper's
 *       method is given for calls).  Priced exactly as the call of the
 *       mirrored lattice: spot K, strike S0, the put's weights times the
 *       child/parent price ratio, read right to left (lattice put-call
 *       symmetry), so the same divider lemma and kernels apply. */
typedef enum {
    AOP_BINOMIAL_CALL = 0,
    AOP_TRINOMIAL_CALL = 1,
    AOP_BSM_PUT = 2,
    AOP_BINOMIAL_PUT = 3,
    AOP_TRINOMIAL_PUT = 4
} aop_model;

typedef enum {
    AOP_OK = 0,
    AOP_EINVAL = 1,      /* bad argument: S0, K, sigma or expiry <= 0, T < 1,
                            T > AOP_MAX_T, unknown model/method, NULL where a
                            pointer is required */
    AOP_EUNSTABLE = 2,   /* a lattice probability or FD weight is negative
                            (binomial p outside [0,1], trinomial p_x < 0,
                            BSM a, b or c < 0) */
    AOP_ENOMEM = 3,      /* workspace cap exceeded or device allocation failed */
    AOP_ECUDA = 4,       /* a CUDA runtime call failed / no usable device */
    AOP_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    AOP_EBUSY = 6,       /* admission refused: no workspace slot free */
    AOP_EINTERNAL = 7,   /* a device-side consistency check failed */
    AOP_ERANGE = 8       /* continuation values of the call reach 1e30 (FP32
                            methods: price it with AOP_FFT_FP64) or 1e300
                            (FP64): node prices far in the money with no early
                            exercise there */
} aop_status;

typedef enum {
    AOP_FFT_FP64 = 0,       /* trapezoidal D&C, FFT convolutions in FP64 */
    AOP_FFT_FP32SPLIT = 1,  /* trapezoidal D&C, FFT convolutions in FP32 on
                               hi/lo split inputs with hi/lo twiddles; base
                               cases and boundary tests in doubled FP32 (see
                               AOP_FFT_DF32), root in FP64 */
    AOP_STENCIL_FP64 = 2,   /* plain Theta(T^2) backward induction (Fig. 1 loop
                               and its trinomial / finite-difference analogues),
                               temporally blocked, FP64 */
    AOP_FFT_DF32 = 3,       /* trapezoidal D&C, FFT convolutions in double-float
                               arithmetic (pairs of FP32 numbers, ~48-bit
                               significands, on the FP32 pipe); base cases and
                               boundary tests likewise (in FP64 where a
                               window's prices span more than e^80); root in
                               FP64 */
    AOP_STENCIL_DF32 = 4    /* the plain loop of AOP_STENCIL_FP64 in double-float
                               arithmetic (~2^-48 relative rounding per row;
                               exercise values clamped to +-1e30, far outside
                               the walk's reach from the root) */
} aop_method;

typedef enum {
    AOP_TRI_BOYLE = 0,  /* u = e^{lambda sigma sqrt(dt)}, probabilities matching
                           the first two moments (Boyle 1986); lambda <= 0
                           selects sqrt(3) */
    AOP_TRI_PAPER = 1   /* Sec. 3: u = e^{sigma sqrt(2 dt)},
                           p_u = ((e^{(r-q)dt/2} - u^{-1/2})/(u^{1/2}-u^{-1/2}))^2,
                           p_d = ((u^{1/2} - e^{(r-q)dt/2})/(u^{1/2}-u^{-1/2}))^2 */
} aop_tri_form;

#define AOP_MAX_T (1 << 20)        /* largest supported step count */
#define AOP_BOUNDARY_NONE_PUT (-2147483647 - 1)   /* INT32_MIN */

/* One pricing request (72 bytes, 8-byte aligned; identical layout on host and
 * device).  Parameters use the paper's notation (Table "Notations"):
 * S = S0, K, R = r, Y = q, V = sigma, E = expiry (in years here). */
typedef struct aop_request {
    int32_t model;      /* aop_model */
    int32_t tri_form;   /* aop_tri_form, trinomial only */
    double S0, K, r, q, sigma, expiry;
    int64_t T;          /* number of time steps, 1 <= T <= AOP_MAX_T */
    double lambda;      /* trinomial stretch for AOP_TRI_BOYLE */
} aop_request;

#define AOP_FLAG_OPTION_TIMES 1   /* record each option's device time (D&C methods) */
/* Calls (FFT methods): the convolutions carry the values tilted by the
 * node-price growth e^{-kappa x} when the exercise boundary lies far above the
 * strike or whole rows are red (automatic), so that rounding follows each
 * cell's own scale.  These two bits force the tilt off or on for every call. */
#define AOP_FLAG_TILT_OFF 2
#define AOP_FLAG_TILT_ON 4
/* D&C placement: in the FP32 modes every option's recursion warp runs on the
 * same SM sub-partition, apart from the convolution warps; this bit spreads
 * them one per sub-partition instead (the FP64 mode always spreads). */
#define AOP_FLAG_SPREAD_WALKERS 8
/* Test of the failure path (D&C methods): no convolution warp takes a task and
 * every device-side wait gives up after 20 ms, so each option ends with
 * AOP_ETIMEOUT and a NaN price; the call returns and the context stays usable.
 * Nothing is faulted or hung.  Not for pricing. */
#define AOP_FLAG_TEST_STALL 16
/* Small D&C batches help by default: spare SMs work for the options in
 * flight (Sec. 2.3: the linear advances of a trapezoid run in parallel with
 * the recursion beside them).  A batch of n options, when the GPU has at least
 * 2n SMs, gets min(3, (SMs - n) / n) helping CTAs per option, every CTA on an
 * SM of its own.  Advances too long for one worker tile go on a board in
 * global memory, where the option's own workers and the helping CTAs (all
 * warps on one advance) take them; CTAs whose options are done help too.
 * Prices and dividers are the same to the bit either way: the same passes and
 * stages run on another SM.  Larger batches, serving sessions and the
 * FP32-split method never help (a helper that shares an SM with an option's
 * recursion slows it more than it saves); this bit turns helping off. */
#define AOP_FLAG_NO_HELP 32

typedef struct aop_options {
    int32_t method;     /* aop_method */
    int32_t base_case;  /* D&C base-case height in rows (2 .. 64, clamped) for every option of the call;
                           0 = the context's tuned pick, else 63 for the lattices and 31 for the
                           BSM put (whose base-case windows are four heights wide); 31 for a
                           batch of three-point lattices only that is small enough to help
                           (AOP_FLAG_NO_HELP) */
    int32_t flags;      /* AOP_FLAG_* bits, 0 for none */
    int32_t ctas_per_sm; /* D&C: options in flight per SM; 0 = as many as fit */
    int32_t lg_tile;    /* D&C: log2 of a worker's shared-memory transform tile, 9 .. 11; 0 = tuned default */
    int32_t radix;      /* D&C: transform stages in radix-4 steps (4) or radix-2 steps (2); 0 = tuned default */
} aop_options;

/* Counters accumulated by the kernels of the last batch call (for roofline
 * accounting).  fft_points counts transform lengths N summed over forward and
 * inverse transforms; conv_inputs counts input cells of the linear advances. */
typedef struct aop_stats {
    int64_t options;
    int64_t convolutions;
    int64_t fft_points;
    int64_t fft_flops;          /* 5 N log2 N per complex transform */
    int64_t conv_inputs;
    int64_t conv_outputs;
    int64_t basecase_cells;     /* FP64 cell updates in naive base cases */
    int64_t stencil_cells;      /* FP64 cell updates of the plain stencil */
    int64_t global_fft_bytes;   /* bytes moved by multi-pass (global) FFT passes */
    double kernel_ms;           /* CUDA-event time of the pricing kernel(s) of the
                                   last batch, measured on their launch stream */
    int64_t walker_wait_ns;     /* D&C: time the recursion warps spent waiting for
                                   linear advances, summed over options */
    int64_t worker_busy_ns;     /* D&C: time the worker warps spent in linear
                                   advances, summed over warps */
    int64_t walker_base_ns;     /* D&C: time the recursion warps spent in the
                                   naive base cases, summed over options */
    int64_t basecase_calls;     /* D&C: naive base cases run */
    int64_t basecase_rows;      /* D&C: rows stepped by the naive base cases */
    int64_t walker_ns;          /* D&C: time from the first recursion step to the
                                   root price, summed over options */
    int64_t spectrum_ns;        /* D&C: time spent evaluating kernel-power spectra
                                   (FP64), summed over the building warps */
    int64_t spectrum_bins;      /* D&C: kernel-power bins evaluated */
    int64_t basecase_loop_cycles;  /* D&C: SM cycles in the call base cases' row loops */
    int64_t basecase_fill_cycles;  /* D&C: SM cycles filling their exercise tables */
    int64_t advance_count_by_log2n[24];  /* D&C: linear advances (worker warps) by
                                            log2 of their transform length */
    int64_t advance_ns_by_log2n[24];     /* ... and the worker time they took */
    int64_t advance_phase_cycles[5];     /* single-tile advances, SM cycles summed over the
                                            worker warps: spectrum lookup, input staging,
                                            forward transform + product, inverse, store */
    int64_t helped_advances;             /* D&C: linear advances run by
                                            CTAs working for another CTA's option */
    int64_t helped_ns;                   /* ... and the worker time they took */
} aop_stats;

typedef struct aop_ctx aop_ctx;

/* Human-readable name of a status code (static string, never NULL). */
const char *aop_status_string(aop_status s);

/* Create a context on CUDA device `device`.  workspace_cap_bytes bounds the
 * device workspace the context may hold (0 = 64 GiB).  The context owns a CUDA
 * stream and lazily grows its workspace up to the cap.  *ctx receives NULL on
 * failure. */
aop_status aop_ctx_create(aop_ctx **ctx, int device, size_t workspace_cap_bytes);

/* Release every device resource of the context.  NULL is accepted. */
aop_status aop_ctx_destroy(aop_ctx *ctx);

/* Price one option (Sec. 2-4), synchronously, with the FP64 FFT method on
 * device 0 using an internal context.  *price_out in currency units. */
aop_status price_american(int model, double S0, double K, double r, double q,
                          double sigma, double expiry, int64_t T, double *price_out);

/* Price one option with explicit method/options.  boundary_out (nullable,
 * host, int32[T+1]) receives the red-green divider of every lattice row:
 *   calls: boundary[i] = largest column j in [0, D i] whose continuation value
 *          is >= its exercise value (Cor. 2.7), -1 if none (D = 1 binomial,
 *          2 trinomial);
 *   binomial/trinomial puts: boundary[i] = largest column j in [0, D i] whose
 *          exercise value exceeds its continuation value, -1 if none;
 *   BSM put: boundary[n] = largest spatial index k in [-(T-n), T-n] whose
 *          exercise value exceeds its continuation value (BSM boundary
 *          theorem), AOP_BOUNDARY_NONE_PUT if none. */
aop_status price_american_ex(const aop_request *req, const aop_options *opt,
                             double *price_out, int32_t *boundary_out);

/* Price n options given in host arrays (the trapezoidal divide-and-conquer of
 * Sec. 2.3, the appendix TOPM algorithm and Sec. 4.3 per option, options
 * independent); returns when prices[] and status[]
 * (both host, length n) are filled.  status may be NULL.  Returns AOP_OK when
 * the batch ran, even if individual options failed (see status[i]); a bad
 * option does not fail the batch.  Copies to and from the device happen inside
 * this call on `stream` (NULL = the context's stream). */
aop_status price_american_batch(aop_ctx *ctx, int64_t n, const aop_request *reqs,
                                const aop_options *opt, double *prices,
                                aop_status *status, void *stream);

/* Price and sensitivities of n options (host arrays, as price_american_batch)
 * with a divide-and-conquer method (AOP_FFT_*; the AOP_STENCIL_* methods give
 * AOP_EINVAL).  greeks (host, double[3n]) receives per option delta (dV/dS0),
 * gamma (d2V/dS0^2) and theta (dV/dt, per year, t calendar time) from the
 * lattice rows next to the root, the standard lattice estimates:
 *   binomial:  delta = (G11 - G10)/(S0 u - S0 d),
 *              gamma = [(G22 - G21)/(S0 u^2 - S0) - (G21 - G20)/(S0 - S0 d^2)]
 *                      / ((S0 u^2 - S0 d^2)/2),
 *              theta = (G21 - G00)/(2 dt);
 *   trinomial: the same centred differences on row 1 (nodes S0 d, S0, S0 u),
 *              theta = (G11 - G00)/dt;
 *   BSM put:   the same on the grid row next to the root (spots S0 e^{-ds},
 *              S0, S0 e^{ds}), theta = K (v^{T-1}_0 - v^T_0)/dt;
 * with dt = expiry/T.  Rows 1-2 are evaluated in FP64 by the kernel that
 * prices the option (the chain stops two rows early); prices agree with
 * price_american_batch to rounding.  Options with T < 3 or a failed status get
 * NaN sensitivities.  The FP32-split method's value error (~1e-6 relative)
 * makes its gamma and theta unreliable; use AOP_FFT_FP64 or AOP_FFT_DF32. */
aop_status price_american_greeks_batch(aop_ctx *ctx, int64_t n, const aop_request *reqs,
                                       const aop_options *opt, double *prices, double *greeks,
                                       aop_status *status, void *stream);

/* Device-resident batch (the same computation as price_american_batch:
 * Sec. 2.3, the appendix TOPM algorithm, Sec. 4.3): d_reqs (aop_request[n]),
 * d_prices (double[n]) and
 * d_status (int32[n], nullable) are device pointers; enqueued on `stream`,
 * returns without waiting.  d_boundary (nullable) is a device int32 array and
 * d_boundary_offsets (device int64[n], required with d_boundary) gives the
 * start of option i's T_i+1 entries in it.  The inputs must stay valid and
 * unmodified until the stream reaches this work. */
aop_status price_american_batch_device(aop_ctx *ctx, int64_t n, const aop_request *d_reqs,
                                       const aop_options *opt, double *d_prices,
                                       int32_t *d_status, int32_t *d_boundary,
                                       const int64_t *d_boundary_offsets, void *stream);

/* Linear advance of one row segment by h steps of a 2- or 3-point stencil
 * (the FFT-based linear-stencil step used inside every trapezoid, Sec. 2.3
 * "Solving a Trapezoid"): for count segments stored back to back in d_in
 * (count*W doubles, device), writes d_out (count*(W - (nw-1)h) doubles):
 *     out[x] = sum_{t=0}^{(nw-1)h} c_t in[x + t],
 * where c is the h-fold self-convolution of the weights w[0..nw-1].
 * method selects AOP_FFT_FP64, AOP_FFT_FP32SPLIT or AOP_FFT_DF32.
 * Synchronous.  Requires 1 <= nw-1, (nw-1)h < W <= 2^20 (else AOP_EINVAL).
 * AOP_ETIMEOUT when a bounded device-side wait gave up; the segments it hit
 * are then NaN. */
aop_status aop_linear_advance_device(aop_ctx *ctx, int method, int nw, const double *w,
                                     int64_t count, int64_t W, int64_t h,
                                     const double *d_in, double *d_out, void *stream);

/* Counters of the kernels launched by the last batch call on this context
 * (synchronizes the context's stream). */
aop_status aop_ctx_get_stats(aop_ctx *ctx, aop_stats *out);

/* European counterparts of the requests (no early exercise): the root value
 * as one T-step linear advance of the expiry payoff, i.e. one FFT convolution
 * with the T-fold power of the stencil evaluated at the root cell (the linear
 * part of the paper's method alone: the appendix on European call options
 * under the binomial model), in FP64 with the
 * node-price tilt so that the payoff row's range (up to e^{+-700}) costs no
 * accuracy.  Host arrays of n; per-request status (AOP_EINVAL also for
 * T > AOP_EUROPEAN_MAX_T).  The method of the context is not used: always
 * FFT_FP64.  AOP_EBUSY while a serving session holds the context. */
#define AOP_EUROPEAN_MAX_T ((int64_t)1 << 19)
aop_status price_european_batch(aop_ctx *ctx, int64_t n, const aop_request *reqs, double *prices,
                                aop_status *status);

/* ---------------------------------------------------------------- serving
 * Continuous pricing of requests as they arrive (no counterpart in the
 * paper, which prices one option per call).  A session runs one persistent
 * pricing kernel: its CTAs -- one option each, as many as the context's
 * workspace cap admits for requests up to T_max steps (aop_server_info) --
 * take the next published request whenever they finish one, so requests that
 * arrive while others are on the GPU start as soon as a slot frees, and
 * short and long options of every model overlap on the device.  Requests and
 * results travel through host memory mapped into the device: no copy or
 * launch per request.  The kernel exits after 2 s without a request and is
 * relaunched by the next call that finds published requests undone.
 *
 * Results are those of price_american_batch with the same options (each
 * request is priced by the same kernel code on its own slot).  While a
 * session lives, the context's batch calls return AOP_EBUSY.  One host thread
 * drives a session at a time.  Errors: AOP_EINVAL (bad arguments; a method
 * other than the three D&C pricers; a request with T > T_max gets that status
 * in its result), AOP_EBUSY (capacity used up, or the context already serves),
 * AOP_ENOMEM, AOP_ECUDA. */
typedef struct aop_server aop_server;

/* Admission planning (a deployment helper; the paper has no counterpart).
 * Device workspace (bytes) that a context's cap must allow for
 * options_in_flight options of up to T_max steps priced at once with a D&C
 * method (AOP_FFT_FP64, AOP_FFT_FP32SPLIT, AOP_FFT_DF32) and base-case height
 * base_case (0 = the library default): the per-option scratch of the
 * divide-and-conquer (current row, per-depth rows, transform scratch, kernel
 * powers) times the count, plus the launch's queue words.  Admission: a
 * serving session on a context created with this cap holds options_in_flight
 * slots for requests up to T_max.  Host-only arithmetic; AOP_EINVAL for a
 * plain stencil method or bad sizes. */
aop_status aop_workspace_bytes(int method, int64_t T_max, int base_case, int64_t options_in_flight,
                               size_t *bytes_out);

/* Start a session on ctx for at most `capacity` requests of up to T_max steps,
 * priced with *opt (method, base case, flags, options per SM; NULL = FFT_FP64
 * defaults). */
aop_status aop_server_create(aop_ctx *ctx, int64_t capacity, int64_t T_max, const aop_options *opt,
                             aop_server **out);
/* Publish one request (copied); *id_out (nullable) receives its index. */
aop_status aop_server_submit(aop_server *srv, const aop_request *req, int64_t *id_out);
/* *done = 1 once request id is priced; then *price and *status (nullable)
 * hold its result. */
aop_status aop_server_poll(aop_server *srv, int64_t id, double *price, aop_status *status, int32_t *done);
/* Replay a recorded stream: publish reqs[i] at arrival_ns[i] nanoseconds (non-
 * decreasing) after the call starts, by the host's steady clock, and return
 * when all n are priced (or AOP_ETIMEOUT timeout_s after the last arrival).
 * latency_ns[i] (nullable) = completion seen by the host - scheduled arrival.
 * prices and status (nullable) are host arrays of n. */
aop_status aop_server_serve_stream(aop_server *srv, int64_t n, const aop_request *reqs,
                                   const int64_t *arrival_ns, double *prices, aop_status *status,
                                   int64_t *latency_ns, double timeout_s);
/* Pricing slots of the session and requests published so far (nullable). */
aop_status aop_server_info(const aop_server *srv, int64_t *slots, int64_t *published);
/* Ask the kernel to stop, wait for the options in flight, free the session. */
aop_status aop_server_destroy(aop_server *srv);

/* Autotuner for the divide-and-conquer methods (no counterpart in the paper,
 * which fixes its base case by hand): prices the n host requests twice per
 * schedule and times each second run with CUDA events.  Stage 1 searches the
 * base-case height in {16, 31, 32, 47, 63, 64} x options in flight per SM in
 * {1, 2, 3, 4} (skipping counts the kernel's registers and shared memory
 * cannot hold) x the transform radix (4, 2) at the default 2^10-value tile;
 * stage 2 tries tiles of 2^9 and 2^11 values at the stage-1 pick; when that
 * moved the tile, stage 3 searches the height x count again at it.  The
 * fastest schedule is kept in this context under the key (method, log2 of
 * the largest T of the requests, model class: binomial
 * only, three-point only, or both) and used by later calls whose aop_options
 * leave a field 0: a call takes the pick of its own key, else of the same size
 * with another model class, else of the nearest size.  best_out (nullable)
 * receives it.  Costs up to 146 batch calls: pass a sample of the workload, or
 * the workload itself when it is priced repeatedly.  AOP_EINVAL for the plain
 * stencil or a bad method. */
aop_status aop_ctx_autotune(aop_ctx *ctx, int64_t n, const aop_request *reqs, int32_t method,
                            aop_options *best_out);
/* aop_ctx_autotune with the candidates' batch calls made with `flags` (AOP_FLAG_*
 * bits): AOP_FLAG_NO_HELP tunes for a use that does not help, such as a
 * serving session, whose requests run without helping CTAs.  The pick is
 * stored under the same key. */
aop_status aop_ctx_autotune_flags(aop_ctx *ctx, int64_t n, const aop_request *reqs, int32_t method,
                                  int32_t flags, aop_options *best_out);

/* The D&C schedule (a tuning aid; the paper has no counterpart) that a batch
 * call with these n host requests and *opt would use on this context: the fields of *opt that are nonzero, the rest from the
 * context's tuned picks (see aop_ctx_autotune) or the library defaults.
 * ctas_per_sm 0 in *out means as many as fit.  Host-only; AOP_EINVAL for a
 * plain stencil method. */
aop_status aop_ctx_schedule(const aop_ctx *ctx, int64_t n, const aop_request *reqs, const aop_options *opt,
                            aop_options *out);

/* Allocation-free variant of aop_linear_advance_device (the paper has no
 * counterpart; this is a deployment convenience).
 *
 * For callers that cannot allocate device memory when they call in: a serving
 * thread held to a fixed memory budget, a host application whose own allocator
 * owns the device memory, code that must not take the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.  It needs no context: its scratch
 * space (FFT work area, kernel-power band, twiddle tables) is one file-scope
 * device array of 7.3 MB (7.0 MiB) that every GPU loading the library keeps until
 * the process exits.  Inputs and outputs are the caller's device buffers, with
 * the same layout and meaning as in aop_linear_advance_device; the call is
 * asynchronous on `stream` (NULL = the legacy default stream) on the current
 * device.
 *
 * Limits: 2 <= W <= AOP_NOALLOC_MAX_W, otherwise AOP_EINVAL (use
 * aop_linear_advance_device for wider segments).  The first call in a CUDA
 * context (per device; again after cudaDeviceReset or any other re-creation
 * of the context, which the call detects by the context's id) looks up the
 * array's device address and fills its twiddle tables, and waits for that on
 * `stream`; make that first call before any stream capture.  Device-side
 * failures are not returned: a segment whose bounded device wait gave up is
 * written as NaN.  All
 * calls share the one array: calls whose kernels overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Nothing is allocated or freed by this call. */
#define AOP_NOALLOC_MAX_W 16384
aop_status aop_linear_advance_noalloc(int method, int nw, const double *w, int64_t count,
                                      int64_t W, int64_t h, const double *d_in, double *d_out,
                                      void *stream);

/* Per-option device time (ns, from the first to the last instruction the
 * pricing kernel spent on the option) of the last D&C batch that was run with
 * AOP_FLAG_OPTION_TIMES; ns_out is a host array of n <= batch size entries.
 * Synchronizes the context.  AOP_EINVAL if the last batch did not record them. */
aop_status aop_ctx_get_option_times(aop_ctx *ctx, int64_t n, int64_t *ns_out);

/* Measured FMA throughput of device `device` (flop/s, two per FMA) for
 * bits = 32 (FP32 pipe) or 64 (FP64 pipe): eight independent FMA chains per
 * thread over 8 CTAs of 256 threads per SM, timed with CUDA events, best of
 * three runs after one warm-up (about 0.1 s each).  A diagnostic for the
 * roofline of the pricer's kernels (the paper has no counterpart).  Blocks
 * the calling thread; AOP_EINVAL for other widths, AOP_ECUDA without a
 * device. */
aop_status aop_measure_fma_peak(int device, int bits, double *flops_per_s);

/* Library version string. */
const char *aop_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AMERICAN_H */
