// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/american.h"

namespace aop {

struct Params;

// Tunables of one batch launch.
struct LaunchCfg {
    int method;          // aop_method
    int base_case;       // D&C base-case height (power of two)
    int64_t T_max;       // largest step count in the batch
    int any_call;        // batch holds at least one binomial/trinomial call
    int any_put;         // batch holds at least one BSM put
};

// Workspace bump allocator over one device buffer owned by the context.
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    void *take(size_t bytes) {
        size_t off = (used + 255) & ~(size_t)255;
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

// setup.cu
cudaError_t launch_params(int64_t n, const aop_request *d_reqs, Params *d_params,
                          int32_t *d_status, int64_t *d_tmax, cudaStream_t s);
cudaError_t launch_twiddles(int log2n, void *d_tw32, void *d_tw64, cudaStream_t s);
// Boundaries of options whose Params have mirror set (binomial and trinomial
// puts priced as mirrored calls): b[i] <- D i - 1 - b[i] for rows 0..T.
cudaError_t launch_mirror_boundaries(int64_t n, const Params *d_params, int32_t *d_bnd,
                                     const int64_t *d_bnd_off, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s);

// stencil.cu -- plain Theta(T^2) lattice loop (temporally blocked)
size_t stencil_workspace_bytes(int64_t n, int64_t T_max);
cudaError_t run_stencil(int64_t n, const Params *d_params, int64_t T_max, void *ws,
                        double *d_prices, int32_t *d_status, int32_t *d_bnd,
                        const int64_t *d_bnd_off, aop_stats *d_stats, cudaStream_t s, bool df);

// dnc.cu / dnc_help.cu -- trapezoidal divide-and-conquer pricer
// log2 of a worker's transform tile unless a schedule says otherwise
constexpr int kDefaultLgTile = 10;
constexpr int kHelpers = 3;     // helping: at most this many extra CTAs per option of a small batch
int dnc_max_per_sm(int method, int64_t T_max, int base_case, int lg_tile = kDefaultLgTile);
// Helping CTAs per option that a batch of n options gets on this device (0: none)
int dnc_helpers(int64_t n, int device);
// per-option workspace of the pricing kernel (one slot), without the
// launch's 8 KiB of queue words
size_t dnc_slot_bytes(int method, int64_t T_max, int base_case);
size_t dnc_workspace_bytes(int method, int64_t n, int64_t T_max, int base_case, int cap, int *grid_out,
                           int device, int lg_tile = kDefaultLgTile, bool help = false);
// A serving session's host-shared state (see aop_server_* in the header):
// requests and results live in mapped host memory, the claim counter on the
// device.  run_dnc with a session prices the published requests in order of
// claim instead of a batch of Params.
struct ServeSession {
    const aop_request *reqs;        // capacity entries (device view of host memory)
    const volatile long long *pub;  // requests published by the host
    const volatile int *stop;       // set by the host to end the kernel
    unsigned long long *claim;      // device counter of claimed requests
    volatile int32_t *done;         // per request: 1 once its result is written
    double *prices;                 // per request (device view of host memory)
    int32_t *status;
    int64_t capacity;
};

cudaError_t run_dnc(int method, int64_t n, const Params *d_params, int64_t T_max, int base_case,
                    void *ws, size_t ws_bytes, const void *d_tw, int tw_log2, double *d_prices,
                    int32_t *d_status, int32_t *d_bnd, const int64_t *d_bnd_off,
                    aop_stats *d_stats, int *d_err, int64_t *d_opt_ns, int flags, int cap, int device,
                    cudaStream_t s, const ServeSession *srv = nullptr, const int32_t *d_order = nullptr,
                    double *d_greeks = nullptr, int lg_tile = kDefaultLgTile, int radix2 = 0,
                    int base_case_put = 0);
cudaError_t run_linear_advance(int method, int nw, const double *w, int64_t count, int64_t W,
                               int64_t h, const double *d_in, double *d_out, const void *d_tw,
                               int tw_log2, void *ws, size_t ws_bytes, int *d_err,
                               cudaStream_t s);
size_t linear_advance_workspace_bytes(int method, int64_t W, int64_t h);
size_t european_workspace_bytes(int64_t n, int64_t T_max, int *grid_out, int device);
cudaError_t run_european(int64_t n, const Params *d_params, int64_t T_max, void *ws, size_t ws_bytes,
                         const void *d_tw, int tw_log2, double *d_prices, int32_t *d_status, int device,
                         cudaStream_t s);

}  // namespace aop
