"""European counterparts by one FFT advance (price_european_batch): against
the oracle's plain backward induction without the max, the binomial sum in
closed form, and the Black-Scholes limit; q = 0 calls equal their American
price (no early exercise)."""
import math

import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import closed_forms as cf
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


def test_against_oracle(ctx):
    reqs = wl.random_small(30, seed=41, T_range=(8, 900))
    prices, status = ctx.price_european(reqs)
    assert (status == 0).all()
    for r, p in zip(reqs, prices):
        ref = oracle.price_european(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(aop.FFT_FP64, ref, r.K), (r, p, ref)


def test_binomial_sum_and_black_scholes_at_large_T(ctx):
    """T = 2^16: the binomial European call equals the closed-form binomial
    sum; all three lattices approach Black-Scholes (error O(1/T) bounded
    here by 2e-3 of the price)."""
    T = 1 << 16
    S, K, r, q, sig, E = 100.0, 95.0, 0.05, 0.02, 0.25, 1.0
    reqs = [wl.Request(0, S, K, r, q, sig, E, T), wl.Request(1, S, K, r, q, sig, E, T, math.sqrt(3)),
            wl.Request(2, S, K, r, 0.0, sig, E, T)]
    prices, status = ctx.price_european(reqs)
    assert (status == 0).all()
    dt = E / T
    u = math.exp(sig * math.sqrt(dt))
    p = (math.exp((r - q) * dt) - 1.0 / u) / (u - 1.0 / u)
    exact = cf.binomial_european_call(S, K, T, u, p, math.exp(-r * dt))
    assert abs(prices[0] - exact) <= 1e-10 * exact + 1e-12 * K, (prices[0], exact)
    assert abs(prices[0] - cf.bs_call(S, K, r, q, sig, E)) <= 2e-3 * prices[0]
    assert abs(prices[1] - cf.bs_call(S, K, r, q, sig, E)) <= 2e-3 * prices[1]
    assert abs(prices[2] - cf.bs_put(S, K, r, 0.0, sig, E)) <= 2e-3 * prices[2]


def test_no_yield_call_equals_american_and_wide_rows(ctx):
    """q = 0: the American call is never exercised early, so both pricers
    agree; sigma 0.6 over three years at T = 8192 spans node prices e^{+-94},
    which the tilted advance carries without loss."""
    reqs = [wl.Request(0, 100.0, 100.0, 0.05, 0.0, 0.6, 3.0, 8192),
            wl.Request(1, 100.0, 110.0, 0.03, 0.0, 0.3, 1.0, 4096, math.sqrt(3))]
    prices, status = ctx.price_european(reqs)
    assert (status == 0).all()
    for r, p in zip(reqs, prices):
        ref = oracle.price_american(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(aop.FFT_FP64, ref, r.K), (r, p, ref)


def test_status(ctx):
    bad = wl.Request(0, -1.0, 100.0, 0.05, 0.02, 0.2, 1.0, 100)
    prices, status = ctx.price_european([bad, wl.fixed_call(0, 64)])
    assert status[0] == 1 and np.isnan(prices[0]) and status[1] == 0
