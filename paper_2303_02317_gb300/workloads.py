"""Seeded synthetic workloads for the American option pricer.

This module holds no pricing arithmetic: it only draws option parameters (and
arrival times) with fixed seeds so that the CUDA library, the tests and the
CPU oracle all see identical inputs.  The paper itself uses one fixed option
(Sec. 5, parameter values) and varies only the step count T; the other
workloads below are synthetic option books with the parameter ranges of the
benchmark configurations.

Model codes: 0 = binomial (CRR) American call, 1 = trinomial American call,
2 = Black-Scholes-Merton explicit finite-difference American put, 3 = binomial
American put, 4 = trinomial American put.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, replace
from typing import List, Tuple

import numpy as np

BINOMIAL_CALL, TRINOMIAL_CALL, BSM_PUT, BINOMIAL_PUT, TRINOMIAL_PUT = 0, 1, 2, 3, 4
TRI_BOYLE, TRI_PAPER = 0, 1
SQRT3 = math.sqrt(3.0)


@dataclass(frozen=True)
class Request:
    model: int
    S0: float
    K: float
    r: float
    q: float
    sigma: float
    expiry: float          # years
    T: int                 # time steps
    lam: float = 0.0       # trinomial stretch (Boyle form); 0 selects sqrt(3)
    tri_form: int = TRI_BOYLE

    def as_dict(self) -> dict:
        return asdict(self)

    def with_T(self, T: int) -> "Request":
        return replace(self, T=int(T))


def single_binomial_t2048() -> Request:
    """Binomial call, S0=K=100, r=0.03, q=0.02, sigma=0.2, 1 year, T=2048."""
    return Request(BINOMIAL_CALL, 100.0, 100.0, 0.03, 0.02, 0.2, 1.0, 2048)


def fixed_call(model: int, T: int, tri_form: int = TRI_BOYLE) -> Request:
    """Binomial or trinomial call at S0=K=100, r=0.05, q=0.03, sigma=0.25,
    1 year (trinomial: Boyle form with lambda=sqrt(3) unless the paper form
    is asked for)."""
    lam = SQRT3 if (model == TRINOMIAL_CALL and tri_form == TRI_BOYLE) else 0.0
    return Request(model, 100.0, 100.0, 0.05, 0.03, 0.25, 1.0, int(T), lam, tri_form)


def fixed_put(model: int, T: int, tri_form: int = TRI_BOYLE) -> Request:
    """Binomial or trinomial put at S0=K=100, r=0.05, q=0.03, sigma=0.25,
    1 year (the fixed call's parameters)."""
    lam = SQRT3 if (model == TRINOMIAL_PUT and tri_form == TRI_BOYLE) else 0.0
    return Request(model, 100.0, 100.0, 0.05, 0.03, 0.25, 1.0, int(T), lam, tri_form)


def fixed_bsm_put(T: int) -> Request:
    """BSM explicit-FD put, S0=K=100, r=0.05, q=0, sigma=0.3, 1 year."""
    return Request(BSM_PUT, 100.0, 100.0, 0.05, 0.0, 0.3, 1.0, int(T))


def paper_params(model: int, T: int) -> Request:
    """The paper's experiment parameters (Sec. 5): E=252 days (252/365 yr),
    K=130, S=127.62, R=0.00163, V=0.2, Y=0.0163 (BSM: Y=0)."""
    q = 0.0 if model == BSM_PUT else 0.0163
    lam = SQRT3 if model == TRINOMIAL_CALL else 0.0
    return Request(model, 127.62, 130.0, 0.00163, q, 0.2, 252.0 / 365.0, int(T), lam)


def _draw_params(rng: np.random.Generator, n: int, put: bool):
    S0 = rng.uniform(50.0, 150.0, n)
    K = rng.uniform(50.0, 150.0, n)
    sigma = rng.uniform(0.1, 0.6, n)
    r = rng.uniform(0.0, 0.08, n)
    q = np.zeros(n) if put else rng.uniform(0.005, 0.06, n)
    expiry = rng.uniform(0.1, 3.0, n)
    return S0, K, sigma, r, q, expiry


def precision_sweep(T: int = 2 ** 17, n_binomial: int = 256, n_trinomial: int = 256,
                    seed: int = 2303) -> List[Request]:
    """Option book of binomial then trinomial calls with S0, K ~ U[50,150],
    sigma ~ U[0.1,0.6], r ~ U[0,0.08], q ~ U[0.005,0.06], expiry ~ U[0.1,3]
    years, all at T steps (trinomial: Boyle form, lambda=sqrt(3))."""
    rng = np.random.default_rng(seed)
    out: List[Request] = []
    for model, n in ((BINOMIAL_CALL, n_binomial), (TRINOMIAL_CALL, n_trinomial)):
        S0, K, sigma, r, q, E = _draw_params(rng, n, put=False)
        lam = SQRT3 if model == TRINOMIAL_CALL else 0.0
        for i in range(n):
            out.append(Request(model, float(S0[i]), float(K[i]), float(r[i]), float(q[i]),
                               float(sigma[i]), float(E[i]), int(T), lam))
    return out


def request_stream(n: int = 65536, rate: float = 20000.0, seed: int = 2317,
                   t_min_log2: float = 10.0, t_max_log2: float = 18.0
                   ) -> Tuple[List[Request], np.ndarray]:
    """Poisson request stream: exponential inter-arrival gaps of mean 1/rate
    seconds; model mix 40% binomial call, 40% trinomial call, 20% BSM put
    (q=0); T = round(2^U[t_min_log2, t_max_log2]); other parameters as in the
    precision sweep.  Returns (requests, arrival times in seconds)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    arrivals = np.cumsum(gaps) - gaps[0]
    u = rng.uniform(0.0, 1.0, n)
    model = np.where(u < 0.4, BINOMIAL_CALL, np.where(u < 0.8, TRINOMIAL_CALL, BSM_PUT))
    T = np.rint(2.0 ** rng.uniform(t_min_log2, t_max_log2, n)).astype(np.int64)
    S0, K, sigma, r, q, E = _draw_params(rng, n, put=False)
    reqs: List[Request] = []
    for i in range(n):
        m = int(model[i])
        reqs.append(Request(m, float(S0[i]), float(K[i]), float(r[i]),
                            0.0 if m == BSM_PUT else float(q[i]), float(sigma[i]),
                            float(E[i]), int(T[i]), SQRT3 if m == TRINOMIAL_CALL else 0.0))
    return reqs, arrivals


def random_small(n: int, seed: int, T_range=(8, 600), models=(0, 1, 2),
                 bsm_yield: bool = False) -> List[Request]:
    """Small mixed cases for parity tests: T uniform in T_range, parameters as
    in the precision sweep, trinomial cases alternate Boyle and paper forms.
    BSM puts have q = 0 unless bsm_yield, which draws q like the lattices."""
    rng = np.random.default_rng(seed)
    out: List[Request] = []
    for i in range(n):
        m = int(models[i % len(models)])
        S0, K, sigma, r, q, E = (float(x[0]) for x in
                                 _draw_params(rng, 1, put=(m == BSM_PUT and not bsm_yield)))
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        if m in (TRINOMIAL_CALL, TRINOMIAL_PUT):
            form = TRI_PAPER if (i // len(models)) % 2 else TRI_BOYLE
            out.append(Request(m, S0, K, r, q, sigma, E, T, SQRT3 if form == TRI_BOYLE else 0.0, form))
        else:
            out.append(Request(m, S0, K, r, q, sigma, E, T))
    return out
