"""The largest supported size, T = AOP_MAX_T = 2^20, through the C ABI, checked
against facts that hold at any size (the oracle's Θ(T²) loop is too slow here):

* a binomial American call without dividends is never exercised early, so it
  equals the European binomial sum, evaluated in closed form (log-space
  weights, node prices as e^{k log u});
* the trinomial call and the BSM put lie between their intrinsic and upper
  bounds and move by less than the lattice's O(1/T) convergence between
  T = 2^19 and 2^20;
* one step more than AOP_MAX_T is rejected with AOP_EINVAL.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import parity

pytestmark = pytest.mark.gpu

T_MAX = 1 << 20


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


def european_binomial_call(req):
    """sum_j C(T,j) p^j (1-p)^(T-j) m^T (S0 e^{(2j-T) log u} - K)^+ with the
    lattice parameters of the oracle.  The binomial probabilities come from
    scipy's binomial distribution (a saddle-point evaluation accurate to a few
    ulps at any T; log-gamma differences of ~1e7 would lose 1e-9 here), and the
    terms are summed exactly."""
    stats = pytest.importorskip("scipy.stats")
    P = oracle.params(req)
    T = req["T"]
    j = np.arange(T + 1)
    pay = req["S0"] * np.exp((2 * j - T) * P["logu"]) - req["K"]
    keep = pay > 0
    w = stats.binom.pmf(j[keep], T, P["p"])
    return math.fsum((w * pay[keep]).tolist()) * math.exp(T * math.log(P["m"]))


def test_binomial_call_without_dividend_at_max_T(ctx):
    """FP64 equals the closed form.  Without a dividend every row is red and
    the node prices reach e^{sigma sqrt(E T)} = e^256 of the spot, past the
    FP32 methods' 1e30 range: they answer AOP_ERANGE (8) instead of a price."""
    req = wl.Request(0, 100.0, 100.0, 0.05, 0.0, 0.25, 1.0, T_MAX).as_dict()
    ref = european_binomial_call(req)
    prices, status = ctx.price_batch([req], method=aop.FFT_FP64)
    assert status[0] == 0
    # The closed form weights each path exactly; any FP64 evaluation of the
    # lattice multiplies T weights that are each rounded (relative 2^-53), so
    # it may sit up to about T * 2^-53 (1.2e-10 at T = 2^20) from it; the
    # oracle's own distance to this sum grows like that (7e-13, 2.8e-12,
    # 1.1e-11 at T = 2^10, 2^12, 2^14).  Tolerance: four times that bound.
    tol = max(parity.price_tol(aop.FFT_FP64, ref, req["K"]), 4 * T_MAX * 2.0 ** -53 * ref)
    assert abs(prices[0] - ref) <= tol, (prices[0], ref, abs(prices[0] - ref) / ref)
    prices, status = ctx.price_batch([req], method=aop.FFT_DF32)
    assert status[0] == 8 and np.isnan(prices[0])


@pytest.mark.parametrize("model", [0, 1, 2], ids=["binomial_call", "trinomial_call", "bsm_put"])
def test_bounds_and_convergence_at_max_T(ctx, model):
    """Doubled FP32 at T = 2^20 (the calls with a 3 % yield, whose green cells
    keep the node prices in range)."""
    base = wl.fixed_call(model, T_MAX) if model < 2 else wl.fixed_bsm_put(T_MAX)
    r = base.as_dict()
    half = dict(r, T=T_MAX // 2)
    prices, status = ctx.price_batch([r, half], method=aop.FFT_DF32)
    assert (status == 0).all()
    p, ph = prices
    S, K = r["S0"], r["K"]
    if model == 2:
        assert max(K - S, 0.0) - 1e-9 * K <= p <= K
    else:
        assert max(S - K, 0.0) - 1e-9 * K <= p <= S
    # the lattices converge like 1/T: doubling T at 2^19 moves the price by far
    # less than 1e-3 of it
    assert abs(p - ph) <= 1e-3 * p, (p, ph)


@pytest.mark.parametrize("method", [aop.FFT_DF32, aop.FFT_FP64, aop.STENCIL_DF32],
                         ids=["df32", "fft64", "stencil_df32"])
def test_one_step_beyond_max_T_is_rejected(ctx, method):
    """Alone (no launch at all) and beside a valid option (rejected inside the
    launch): AOP_EINVAL (1) and a NaN price, the valid option priced."""
    r = wl.fixed_call(0, T_MAX + 1).as_dict()
    prices, status = ctx.price_batch([r, r], method=method)
    assert (status == 1).all() and np.isnan(prices).all(), (status, prices)
    ok = wl.fixed_call(0, 1024).as_dict()
    prices, status = ctx.price_batch([r, ok], method=method)
    assert list(status) == [1, 0] and np.isnan(prices[0]) and np.isfinite(prices[1]), (status, prices)
