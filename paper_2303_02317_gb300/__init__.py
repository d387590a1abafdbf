"""GB300 (sm_103a) nonlinear-stencil American option pricer.

A thin ctypes binding over the C ABI declared in ``include/american.h``
(``libamerican.so``).  Every pricing step runs in the library's CUDA kernels;
this module only marshals arguments.  If the shared library is missing or no
CUDA device is usable the calls raise -- there is no CPU fallback.

Method codes: FFT_FP64 (trapezoidal divide-and-conquer with FP64 FFT
convolutions and FP64 base cases), FFT_FP32SPLIT (the same with FP32
hi/lo-split convolutions), FFT_DF32 (doubled-FP32 convolutions; both FP32
methods evaluate base cases in doubled FP32, in FP64 where the exercise
values span too wide a range), STENCIL_FP64 (plain Theta(T^2) backward
induction) and STENCIL_DF32 (the same loop in doubled FP32).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Iterable, List, Optional, Sequence

import numpy as np

from .workloads import Request  # noqa: F401  (re-exported for callers)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamerican.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "american.h")

BINOMIAL_CALL, TRINOMIAL_CALL, BSM_PUT, BINOMIAL_PUT, TRINOMIAL_PUT = 0, 1, 2, 3, 4
FFT_FP64, FFT_FP32SPLIT, STENCIL_FP64, FFT_DF32, STENCIL_DF32 = 0, 1, 2, 3, 4
TRI_BOYLE, TRI_PAPER = 0, 1
BOUNDARY_NONE_PUT = -(2 ** 31)
MAX_T = 1 << 20
STATUS = {0: "AOP_OK", 1: "AOP_EINVAL", 2: "AOP_EUNSTABLE", 3: "AOP_ENOMEM",
          4: "AOP_ECUDA", 5: "AOP_ETIMEOUT", 6: "AOP_EBUSY", 7: "AOP_EINTERNAL", 8: "AOP_ERANGE"}

REQUEST_DTYPE = np.dtype([("model", "<i4"), ("tri_form", "<i4"), ("S0", "<f8"), ("K", "<f8"),
                          ("r", "<f8"), ("q", "<f8"), ("sigma", "<f8"), ("expiry", "<f8"),
                          ("T", "<i8"), ("lambda", "<f8")], align=True)
assert REQUEST_DTYPE.itemsize == 72


class AopError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__("%s (%s)%s" % (STATUS.get(self.code, "status %d" % code),
                                        status_string(self.code) if _lib_or_none() else "",
                                        (": " + what) if what else ""))


class _Options(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("base_case", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("lg_tile", ctypes.c_int32), ("radix", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "options", "convolutions", "fft_points", "fft_flops", "conv_inputs", "conv_outputs",
        "basecase_cells", "stencil_cells", "global_fft_bytes")] + [("kernel_ms", ctypes.c_double)] + [
        ("walker_wait_ns", ctypes.c_int64), ("worker_busy_ns", ctypes.c_int64),
        ("walker_base_ns", ctypes.c_int64), ("basecase_calls", ctypes.c_int64),
        ("basecase_rows", ctypes.c_int64), ("walker_ns", ctypes.c_int64),
        ("spectrum_ns", ctypes.c_int64), ("spectrum_bins", ctypes.c_int64),
        ("basecase_loop_cycles", ctypes.c_int64), ("basecase_fill_cycles", ctypes.c_int64),
        ("advance_count_by_log2n", ctypes.c_int64 * 24), ("advance_ns_by_log2n", ctypes.c_int64 * 24),
        ("advance_phase_cycles", ctypes.c_int64 * 5), ("helped_advances", ctypes.c_int64),
        ("helped_ns", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def _lib_or_none():
    return _lib


def load(path: Optional[str] = None):
    """Load libamerican.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("libamerican.so not found at %s; run "
                               "paper_2303_02317_gb300.build.build() (needs nvcc)" % p)
        lib = ctypes.CDLL(p)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.aop_status_string.restype = ctypes.c_char_p
        lib.aop_status_string.argtypes = [ctypes.c_int]
        lib.aop_version.restype = ctypes.c_char_p
        lib.aop_ctx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]
        lib.aop_ctx_destroy.argtypes = [vp]
        lib.price_american.argtypes = [ctypes.c_int, dbl, dbl, dbl, dbl, dbl, dbl, i64,
                                       ctypes.POINTER(dbl)]
        lib.price_american_ex.argtypes = [vp, ctypes.POINTER(_Options), ctypes.POINTER(dbl), vp]
        lib.price_american_batch.argtypes = [vp, i64, vp, ctypes.POINTER(_Options), vp, vp, vp]
        lib.price_american_greeks_batch.argtypes = [vp, i64, vp, ctypes.POINTER(_Options), vp, vp, vp, vp]
        lib.price_american_batch_device.argtypes = [vp, i64, vp, ctypes.POINTER(_Options), vp,
                                                    vp, vp, vp, vp]
        lib.aop_linear_advance_device.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, i64, i64,
                                                  i64, vp, vp, vp]
        lib.aop_ctx_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
        lib.aop_ctx_get_option_times.argtypes = [vp, i64, vp]
        lib.aop_ctx_autotune.argtypes = [vp, i64, vp, i32, ctypes.POINTER(_Options)]
        lib.aop_ctx_autotune_flags.argtypes = [vp, i64, vp, i32, i32, ctypes.POINTER(_Options)]
        lib.price_european_batch.argtypes = [vp, i64, vp, vp, vp]
        lib.aop_server_create.argtypes = [vp, i64, i64, ctypes.POINTER(_Options), ctypes.POINTER(vp)]
        lib.aop_server_submit.argtypes = [vp, vp, ctypes.POINTER(i64)]
        lib.aop_server_poll.argtypes = [vp, i64, ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(i32)]
        lib.aop_server_serve_stream.argtypes = [vp, i64, vp, vp, vp, vp, vp, dbl]
        lib.aop_server_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.aop_server_destroy.argtypes = [vp]
        lib.aop_linear_advance_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, i64, i64, i64,
                                                   vp, vp, vp]
        lib.aop_linear_advance_noalloc.restype = ctypes.c_int
        lib.aop_ctx_schedule.argtypes = [vp, i64, vp, ctypes.POINTER(_Options), ctypes.POINTER(_Options)]
        lib.aop_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(dbl)]
        lib.aop_workspace_bytes.argtypes = [ctypes.c_int, i64, ctypes.c_int, i64, ctypes.POINTER(ctypes.c_size_t)]
        for f in ("aop_ctx_get_option_times", "aop_ctx_create", "aop_ctx_destroy", "price_american", "price_american_ex",
                  "price_american_batch", "price_american_batch_device", "price_american_greeks_batch",
                  "aop_linear_advance_device", "aop_ctx_get_stats", "aop_ctx_autotune",
                  "aop_server_create", "aop_server_submit", "aop_server_poll", "aop_server_serve_stream",
                  "aop_server_info", "aop_server_destroy", "price_european_batch", "aop_workspace_bytes",
                  "aop_measure_fma_peak", "aop_ctx_schedule", "aop_ctx_autotune_flags"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def declared_symbols() -> List[str]:
    """Names of the functions declared in include/american.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       txt, flags=re.M)
    return [n for n in names if n not in ("if", "while", "for", "return")]


def status_string(code: int) -> str:
    return load().aop_status_string(int(code)).decode()


def version() -> str:
    return load().aop_version().decode()


def _check(code: int, what: str = ""):
    if code != 0:
        raise AopError(code, what)


FLAG_OPTION_TIMES = 1
FLAG_TILT_OFF = 2
FLAG_TILT_ON = 4
FLAG_SPREAD_WALKERS = 8
FLAG_TEST_STALL = 16
FLAG_NO_HELP = 32



def _opts(method: int, base_case: int = 0, flags: int = 0, ctas_per_sm: int = 0, lg_tile: int = 0,
          radix: int = 0) -> _Options:
    return _Options(int(method), int(base_case), int(flags), int(ctas_per_sm), int(lg_tile), int(radix))


def requests_array(reqs: Iterable) -> np.ndarray:
    """Pack requests (workloads.Request, dicts or tuples) into aop_request[]."""
    reqs = list(reqs)
    a = np.zeros(len(reqs), dtype=REQUEST_DTYPE)
    for i, r in enumerate(reqs):
        g = (lambda k, d=0: r.get(k, d)) if isinstance(r, dict) else (lambda k, d=0: getattr(r, k, d))
        a[i] = (int(g("model")), int(g("tri_form", 0) or 0), float(g("S0")), float(g("K")),
                float(g("r")), float(g("q")), float(g("sigma")), float(g("expiry")), int(g("T")),
                float(g("lam", 0.0) or 0.0))
    return a


def price_american(model: int, S0: float, K: float, r: float, q: float, sigma: float,
                   expiry: float, T: int) -> float:
    """One option, FP64 FFT method, device 0 (C: price_american)."""
    out = ctypes.c_double()
    _check(load().price_american(int(model), S0, K, r, q, sigma, expiry, int(T), ctypes.byref(out)))
    return out.value


def price_american_ex(req, method: int = FFT_FP64, base_case: int = 0, boundary: bool = False,
                      flags: int = 0):
    """One option with explicit method; returns price or (price, boundary[T+1])."""
    arr = requests_array([req])
    out = ctypes.c_double()
    T = int(arr["T"][0])
    b = np.empty(T + 1, dtype=np.int32) if boundary else None
    o = _opts(method, base_case, flags)
    code = load().price_american_ex(arr.ctypes.data, ctypes.byref(o), ctypes.byref(out),
                                    b.ctypes.data if b is not None else None)
    _check(code, "price_american_ex")
    return (out.value, b) if boundary else out.value


NOALLOC_MAX_W = 16384


def measure_fma_peak(bits: int = 32, device: int = 0) -> float:
    """C: aop_measure_fma_peak -- measured FMA rate (flop/s) of the FP32
    (bits=32) or FP64 (bits=64) pipe of the device."""
    out = ctypes.c_double()
    _check(load().aop_measure_fma_peak(int(device), int(bits), ctypes.byref(out)), "aop_measure_fma_peak")
    return float(out.value)


def workspace_bytes(method: int, T_max: int, options_in_flight: int, base_case: int = 0) -> int:
    """C: aop_workspace_bytes -- the workspace cap that holds options_in_flight
    options of up to T_max steps at once (host arithmetic, no device needed)."""
    out = ctypes.c_size_t()
    _check(load().aop_workspace_bytes(int(method), ctypes.c_int64(int(T_max)), int(base_case),
                                      ctypes.c_int64(int(options_in_flight)), ctypes.byref(out)),
           "aop_workspace_bytes")
    return int(out.value)


def linear_advance_noalloc(method: int, w: Sequence[float], count: int, W: int, h: int,
                           d_in: int, d_out: int, stream: int = 0):
    """C: aop_linear_advance_noalloc -- the linear advance without a context
    and without any device allocation at call time, for callers that cannot
    allocate (fixed memory budget, foreign allocator owning the device memory,
    no implicit synchronisation allowed).  Its scratch is one static device
    array shared by every call: overlapping calls race.  W <= NOALLOC_MAX_W.
    Asynchronous on `stream` (0 = the legacy default stream)."""
    wa = (ctypes.c_double * 3)(*(list(w) + [0.0] * (3 - len(w))))
    _check(load().aop_linear_advance_noalloc(int(method), len(w), wa, int(count), int(W), int(h),
                                             ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                                             ctypes.c_void_p(stream) if stream else None),
           "aop_linear_advance_noalloc")


class Context:
    """An aop_ctx: a device, a stream and a capped workspace."""

    def __init__(self, device: int = 0, workspace_cap_bytes: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.aop_ctx_create(ctypes.byref(h), int(device), ctypes.c_size_t(workspace_cap_bytes)),
               "aop_ctx_create")
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().aop_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # host buffers in, host buffers out (C: price_american_batch)
    def price_batch(self, reqs, method: int = FFT_FP64, base_case: int = 0, stream: int = 0,
                    flags: int = 0, ctas_per_sm: int = 0, lg_tile: int = 0, radix: int = 0):
        arr = reqs if isinstance(reqs, np.ndarray) else requests_array(reqs)
        n = len(arr)
        prices = np.empty(n, dtype=np.float64)
        status = np.empty(n, dtype=np.int32)
        o = _opts(method, base_case, flags, ctas_per_sm, lg_tile, radix)
        _check(load().price_american_batch(self._h, n, arr.ctypes.data, ctypes.byref(o),
                                           prices.ctypes.data, status.ctypes.data,
                                           ctypes.c_void_p(stream) if stream else None),
               "price_american_batch")
        return prices, status

    def price_greeks(self, reqs, method: int = FFT_FP64, base_case: int = 0, stream: int = 0,
                     flags: int = 0, ctas_per_sm: int = 0):
        """Prices and (delta, gamma, theta) per option from the lattice rows
        next to the root (C: price_american_greeks_batch); returns
        (prices[n], greeks[n, 3], status[n])."""
        arr = reqs if isinstance(reqs, np.ndarray) else requests_array(reqs)
        n = len(arr)
        prices = np.empty(n, dtype=np.float64)
        greeks = np.empty((n, 3), dtype=np.float64)
        status = np.empty(n, dtype=np.int32)
        o = _opts(method, base_case, flags, ctas_per_sm)
        _check(load().price_american_greeks_batch(self._h, n, arr.ctypes.data, ctypes.byref(o),
                                                  prices.ctypes.data, greeks.ctypes.data,
                                                  status.ctypes.data,
                                                  ctypes.c_void_p(stream) if stream else None),
               "price_american_greeks_batch")
        return prices, greeks, status

    # device pointers (C: price_american_batch_device)
    def price_batch_device(self, n: int, d_reqs: int, d_prices: int, d_status: int = 0,
                           d_boundary: int = 0, d_boundary_offsets: int = 0,
                           method: int = FFT_FP64, base_case: int = 0, stream: int = 0,
                           flags: int = 0, ctas_per_sm: int = 0, lg_tile: int = 0, radix: int = 0):
        o = _opts(method, base_case, flags, ctas_per_sm, lg_tile, radix)
        _check(load().price_american_batch_device(
            self._h, int(n), ctypes.c_void_p(d_reqs), ctypes.byref(o), ctypes.c_void_p(d_prices),
            ctypes.c_void_p(d_status) if d_status else None,
            ctypes.c_void_p(d_boundary) if d_boundary else None,
            ctypes.c_void_p(d_boundary_offsets) if d_boundary_offsets else None,
            ctypes.c_void_p(stream) if stream else None), "price_american_batch_device")

    def linear_advance_device(self, method: int, w: Sequence[float], count: int, W: int, h: int,
                              d_in: int, d_out: int, stream: int = 0):
        wa = (ctypes.c_double * 3)(*(list(w) + [0.0] * (3 - len(w))))
        _check(load().aop_linear_advance_device(self._h, int(method), len(w), wa, int(count), int(W),
                                                int(h), ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                                                ctypes.c_void_p(stream) if stream else None),
               "aop_linear_advance_device")

    def price_european(self, reqs):
        """European counterparts by one FFT advance each (C: price_european_batch);
        returns (prices, status)."""
        arr = reqs if isinstance(reqs, np.ndarray) else requests_array(reqs)
        n = len(arr)
        prices = np.empty(n, dtype=np.float64)
        status = np.empty(n, dtype=np.int32)
        _check(load().price_european_batch(self._h, n, arr.ctypes.data, prices.ctypes.data, status.ctypes.data),
               "price_european_batch")
        return prices, status

    def autotune(self, reqs, method: int, flags: int = 0) -> dict:
        """Pick this context's D&C schedule (base-case height, options in
        flight per SM, transform tile and radix) for `method` and the size and
        model class of these requests by timing them, the batch calls made
        with `flags` (FLAG_NO_HELP for a serving session's schedule; C:
        aop_ctx_autotune / aop_ctx_autotune_flags)."""
        arr = reqs if isinstance(reqs, np.ndarray) else requests_array(reqs)
        best = _Options()
        if flags:
            _check(load().aop_ctx_autotune_flags(self._h, len(arr), arr.ctypes.data, int(method), int(flags),
                                                 ctypes.byref(best)), "aop_ctx_autotune_flags")
        else:
            _check(load().aop_ctx_autotune(self._h, len(arr), arr.ctypes.data, int(method), ctypes.byref(best)),
                   "aop_ctx_autotune")
        return {"base_case": int(best.base_case), "ctas_per_sm": int(best.ctas_per_sm),
                "lg_tile": int(best.lg_tile), "radix": int(best.radix)}

    def schedule(self, reqs, method: int) -> dict:
        """The D&C schedule a batch of these requests would use on this
        context (C: aop_ctx_schedule)."""
        arr = reqs if isinstance(reqs, np.ndarray) else requests_array(reqs)
        o = _opts(method)
        out = _Options()
        _check(load().aop_ctx_schedule(self._h, len(arr), arr.ctypes.data, ctypes.byref(o), ctypes.byref(out)),
               "aop_ctx_schedule")
        return {"base_case": int(out.base_case), "ctas_per_sm": int(out.ctas_per_sm),
                "lg_tile": int(out.lg_tile), "radix": int(out.radix)}

    def option_times_ns(self, n: int) -> np.ndarray:
        out = np.empty(int(n), dtype=np.int64)
        _check(load().aop_ctx_get_option_times(self._h, int(n), out.ctypes.data),
               "aop_ctx_get_option_times")
        return out

    def stats(self) -> dict:
        s = _Stats()
        _check(load().aop_ctx_get_stats(self._h, ctypes.byref(s)), "aop_ctx_get_stats")
        out = {}
        for k, _ in _Stats._fields_:
            v = getattr(s, k)
            out[k] = float(v) if k == "kernel_ms" else ([int(x) for x in v] if hasattr(v, "__len__") else int(v))
        return out


class Server:
    """Continuous pricing session on a context (C: aop_server_*): one
    persistent pricing kernel takes requests as they are published."""

    def __init__(self, ctx: "Context", capacity: int, T_max: int, method: int = FFT_FP64,
                 base_case: int = 0, flags: int = 0, ctas_per_sm: int = 0, lg_tile: int = 0, radix: int = 0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        o = _opts(method, base_case, flags, ctas_per_sm, lg_tile, radix)
        _check(load().aop_server_create(ctx._h, int(capacity), int(T_max), ctypes.byref(o), ctypes.byref(h)),
               "aop_server_create")
        self._h = h

    def submit(self, req) -> int:
        arr = requests_array([req])
        i = ctypes.c_int64()
        _check(load().aop_server_submit(self._h, arr.ctypes.data, ctypes.byref(i)), "aop_server_submit")
        return int(i.value)

    def poll(self, i: int):
        """(done, price, status) of request i."""
        p, st, d = ctypes.c_double(), ctypes.c_int(), ctypes.c_int32()
        _check(load().aop_server_poll(self._h, int(i), ctypes.byref(p), ctypes.byref(st), ctypes.byref(d)),
               "aop_server_poll")
        return bool(d.value), float(p.value), int(st.value)

    def serve_stream(self, reqs, arrival_s, timeout_s: float = 600.0):
        """Replay requests at their arrival times (seconds from now); returns
        (prices, status, latency seconds)."""
        arr = reqs if isinstance(reqs, np.ndarray) else requests_array(reqs)
        n = len(arr)
        arrival_ns = np.ascontiguousarray(np.rint(np.asarray(arrival_s, dtype=np.float64) * 1e9).astype(np.int64))
        prices = np.empty(n, dtype=np.float64)
        status = np.empty(n, dtype=np.int32)
        lat = np.empty(n, dtype=np.int64)
        _check(load().aop_server_serve_stream(self._h, n, arr.ctypes.data, arrival_ns.ctypes.data,
                                              prices.ctypes.data, status.ctypes.data, lat.ctypes.data,
                                              float(timeout_s)), "aop_server_serve_stream")
        return prices, status, lat / 1e9

    def info(self) -> dict:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().aop_server_info(self._h, ctypes.byref(a), ctypes.byref(b)), "aop_server_info")
        return {"slots": int(a.value), "published": int(b.value)}

    def close(self):
        if getattr(self, "_h", None):
            load().aop_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
