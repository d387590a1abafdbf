"""Plain FP64 CPU oracle for the American option lattices of arXiv 2303.02317.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and the library never imports it.

The C source (``oracle.c``) is the plain definition the fast method must
reproduce: Fig. 1's nested loop for the binomial call (Sec. 2.1, Def. 2.1), the
trinomial call of Sec. 3 and its appendix, the same two lattices with the put's
exercise value, and the explicit finite-difference scheme for the
Black-Scholes-Merton put of Sec. 4 (with an optional dividend yield).  This
wrapper only marshals arguments through ctypes.

Requests are plain mappings (or objects with attributes) with the fields
``model, S0, K, r, q, sigma, expiry, T`` and optionally ``lam`` and
``tri_form``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_oracle.so")

BOPM, TOPM, BSM, BOPM_PUT, TOPM_PUT = 0, 1, 2, 3, 4
OK, EINVAL, EUNSTABLE, ENOMEM = 0, 1, 2, 3
INT32_MIN = -(2 ** 31)


class _Req(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("tri_form", ctypes.c_int32),
        ("S", ctypes.c_double),
        ("K", ctypes.c_double),
        ("R", ctypes.c_double),
        ("Y", ctypes.c_double),
        ("V", ctypes.c_double),
        ("E", ctypes.c_double),
        ("T", ctypes.c_int64),
        ("lam", ctypes.c_double),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("D", ctypes.c_int32),
        ("w", ctypes.c_double * 3),
        ("o_min", ctypes.c_int32),
        ("nw", ctypes.c_int32),
        ("u", ctypes.c_double),
        ("logu", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("dtau", ctypes.c_double),
        ("ds", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("p", ctypes.c_double),
        ("pu", ctypes.c_double),
        ("po", ctypes.c_double),
        ("pd", ctypes.c_double),
        ("m", ctypes.c_double),
        ("omega_y", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so with gcc (OpenMP, no FP contraction so
    that x86 and Arm hosts round every operation as written)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB)
            lib.or_params_compute.argtypes = [ctypes.POINTER(_Req), ctypes.POINTER(_Params)]
            lib.or_price_american.argtypes = [ctypes.POINTER(_Req), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_void_p, ctypes.c_void_p]
            lib.or_price_european.argtypes = [ctypes.POINTER(_Req), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double)]
            lib.or_grid.argtypes = [ctypes.POINTER(_Req), ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p]
            lib.or_greeks.argtypes = [ctypes.POINTER(_Req), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]
            lib.or_price_many.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p]
            lib.or_max_threads.restype = ctypes.c_int
            lib.or_sizeof_req.restype = ctypes.c_int
            assert lib.or_sizeof_req() == ctypes.sizeof(_Req)
            _lib = lib
    return _lib


def _field(req, name, default=None):
    if isinstance(req, dict):
        return req.get(name, default)
    return getattr(req, name, default)


def _to_c(req) -> _Req:
    lam = _field(req, "lam", 0.0)
    return _Req(int(_field(req, "model")), int(_field(req, "tri_form", 0) or 0),
                float(_field(req, "S0")), float(_field(req, "K")), float(_field(req, "r")),
                float(_field(req, "q")), float(_field(req, "sigma")),
                float(_field(req, "expiry")), int(_field(req, "T")),
                float(lam if lam is not None else 0.0))


def columns(req) -> int:
    """Number of stored columns of the widest row: T+1 (BOPM) or 2T+1."""
    T = int(_field(req, "T"))
    return T + 1 if int(_field(req, "model")) in (BOPM, BOPM_PUT) else 2 * T + 1


def params(req) -> dict:
    """Lattice parameters (Sec. 2.1, Sec. 3, Sec. 4); raises on bad input."""
    lib = _load()
    P = _Params()
    st = lib.or_params_compute(ctypes.byref(_to_c(req)), ctypes.byref(P))
    if st:
        raise ValueError("oracle rejected request (status %d)" % st)
    return {"model": P.model, "D": P.D, "w": [P.w[i] for i in range(P.nw)],
            "o_min": P.o_min, "u": P.u, "logu": P.logu, "dt": P.dt, "dtau": P.dtau, "ds": P.ds,
            "omega": P.omega, "omega_y": P.omega_y, "p": P.p, "pu": P.pu, "po": P.po, "pd": P.pd, "m": P.m}


def status_of(req) -> int:
    lib = _load()
    P = _Params()
    return int(lib.or_params_compute(ctypes.byref(_to_c(req)), ctypes.byref(P)))


def price_american(req, nthreads: int = 1, with_boundary: bool = False,
                   with_margin: bool = False):
    """American price by plain backward induction.  Returns ``price`` or
    ``(price, boundary[T+1], margin[T+1])`` when boundary/margin are asked."""
    lib = _load()
    T = int(_field(req, "T"))
    b = np.empty(T + 1, dtype=np.int32) if with_boundary else None
    m = np.empty(T + 1, dtype=np.float64) if with_margin else None
    out = ctypes.c_double()
    st = lib.or_price_american(ctypes.byref(_to_c(req)), int(nthreads), ctypes.byref(out),
                               b.ctypes.data if b is not None else None,
                               m.ctypes.data if m is not None else None)
    if st:
        raise ValueError("oracle status %d" % st)
    if with_boundary or with_margin:
        return out.value, b, m
    return out.value


def price_european(req, nthreads: int = 1) -> float:
    """The same lattice without the early-exercise max."""
    lib = _load()
    out = ctypes.c_double()
    st = lib.or_price_european(ctypes.byref(_to_c(req)), int(nthreads), ctypes.byref(out))
    if st:
        raise ValueError("oracle status %d" % st)
    return out.value


def grid(req, american: bool = True):
    """Every row of the lattice (small T only).  Lattices: shape (T+1, D*T+1),
    entry [i, j]; BSM put: shape (T+1, 2T+1), entry [n, k+T].  Cells outside a
    row are NaN.  Also returns the boundary array."""
    lib = _load()
    T = int(_field(req, "T"))
    g = np.empty((T + 1, columns(req)), dtype=np.float64)
    b = np.empty(T + 1, dtype=np.int32)
    st = lib.or_grid(ctypes.byref(_to_c(req)), 1 if american else 0, g.ctypes.data, b.ctypes.data)
    if st:
        raise ValueError("oracle status %d" % st)
    return g, b


def greeks(req, american: bool = True, nthreads: int = 1):
    """(price, delta, gamma, theta) from the nodes next to the root, and those
    nodes' values: lattices: row 1 at [0:D+1], row 2 at [3:3+2D+1]; BSM put:
    row T-1 (k = -1..1) at [0:3], row T-2 (k = -2..2) at [3:8] (units of K).
    T >= 3."""
    lib = _load()
    out = np.empty(4, dtype=np.float64)
    near = np.full(8, np.nan, dtype=np.float64)
    st = lib.or_greeks(ctypes.byref(_to_c(req)), 1 if american else 0, int(nthreads),
                       out.ctypes.data, near.ctypes.data)
    if st:
        raise ValueError("oracle status %d" % st)
    return tuple(float(x) for x in out), near


def price_many(reqs, nthreads: int = 0):
    """Price a list of requests one after another (OpenMP over each row when
    nthreads != 1; 0 = all cores).  Returns (prices, status)."""
    lib = _load()
    arr = (_Req * len(reqs))(*[_to_c(r) for r in reqs])
    prices = np.empty(len(reqs), dtype=np.float64)
    status = np.empty(len(reqs), dtype=np.int32)
    lib.or_price_many(len(reqs), ctypes.cast(arr, ctypes.c_void_p), int(nthreads),
                      prices.ctypes.data, status.ctypes.data)
    return prices, status


def max_threads() -> int:
    return int(_load().or_max_threads())


def linear_advance(x, w, h: int):
    """The linear stencil of the continuation region applied h times (the
    step each FFT convolution of Sec. 2.3 "Solving a Trapezoid" performs over
    the red cells): y_{k+1}[j] = sum_o w[o] y_k[j + o] for o = 0 .. len(w)-1,
    keeping the cells whose dependency cone lies inside the segment, so that a
    row of W cells yields W - (len(w) - 1) h cells.  Plain FP64 numpy, one
    step at a time.  x: (count, W) or (W,) array."""
    y = np.array(x, dtype=np.float64, copy=True)
    w = [float(v) for v in w]
    span = len(w) - 1
    for _ in range(int(h)):
        n = y.shape[-1] - span
        z = w[0] * y[..., 0:n]
        for o in range(1, span + 1):
            z = z + w[o] * y[..., o:o + n]
        y = z
    return y


def tie_band(req) -> float:
    """Rows whose oracle margin is at most this may legitimately disagree on
    the boundary index by one (a tie between continuation and exercise)."""
    return 1e-12 * (1.0 if int(_field(req, "model")) == BSM else float(_field(req, "K")))


__all__ = ["build", "params", "status_of", "price_american", "price_european", "grid", "greeks", "linear_advance",
           "price_many", "max_threads", "columns", "tie_band", "BOPM", "TOPM", "BSM",
           "BOPM_PUT", "TOPM_PUT", "INT32_MIN"]
