"""Sensitivities (delta, gamma, theta) from the rows next to the root,
through the C ABI (price_american_greeks_batch), against the CPU oracle's
values from its own backward induction.  Tolerances follow from the price
tolerance tp of the method: a difference of two node values over a spot step
h1 = S0 (e^l - e^-l) (l the log step of the lattice) gives delta within
4 tp / h1, gamma within 16 tp / h1^2 and theta within 4 tp / dt."""
import math

import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import parity

pytestmark = pytest.mark.gpu

MODELS = (aop.BINOMIAL_CALL, aop.TRINOMIAL_CALL, aop.BSM_PUT, aop.BINOMIAL_PUT, aop.TRINOMIAL_PUT)


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


def _check(method, reqs, prices, greeks, status):
    assert (status == 0).all(), status
    for r, p, g in zip(reqs, prices, greeks):
        d = r.as_dict()
        (op, od, og, ot), _ = oracle.greeks(d)
        P = oracle.params(d)
        tp = parity.price_tol(method, op, max(r.K, r.S0))
        ell = P["ds"] if r.model == aop.BSM_PUT else P["logu"]
        h1 = r.S0 * (math.exp(ell) - math.exp(-ell))
        dt = r.expiry / r.T
        assert abs(p - op) <= tp, (r, p, op)
        assert abs(g[0] - od) <= 4 * tp / h1, (r, "delta", g[0], od)
        assert abs(g[1] - og) <= 16 * tp / h1 ** 2, (r, "gamma", g[1], og)
        assert abs(g[2] - ot) <= 4 * tp / dt, (r, "theta", g[2], ot)


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_DF32], ids=["fft64", "df32"])
def test_greeks_random(ctx, method):
    reqs = wl.random_small(40, seed=51, T_range=(3, 900), models=MODELS, bsm_yield=True)
    prices, greeks, status = ctx.price_greeks(reqs, method=method)
    _check(method, reqs, prices, greeks, status)
    # the same prices as the plain batch, to rounding
    plain, st = ctx.price_batch(reqs, method=method)
    assert (st == 0).all()
    for r, a, b in zip(reqs, prices, plain):
        assert abs(a - b) <= parity.price_tol(method, b, max(r.K, r.S0))


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_DF32], ids=["fft64", "df32"])
@pytest.mark.parametrize("B", [2, 16, 64])
def test_greeks_base_case_heights_and_mid_size(ctx, method, B):
    reqs = [wl.fixed_call(0, 5000), wl.fixed_call(1, 3001), wl.fixed_bsm_put(4000),
            wl.fixed_put(aop.BINOMIAL_PUT, 4097), wl.fixed_put(aop.TRINOMIAL_PUT, 2500, wl.TRI_PAPER),
            wl.Request(2, 100.0, 100.0, 0.05, 0.03, 0.3, 1.0, 3000),
            # exercised at the root: every node next to it green
            wl.Request(aop.BINOMIAL_PUT, 40.0, 150.0, 0.08, 0.0, 0.15, 2.0, 600),
            wl.Request(aop.BINOMIAL_CALL, 150.0, 50.0, 0.01, 0.08, 0.15, 2.0, 600),
            wl.Request(2, 50.0, 150.0, 0.08, 0.0, 0.2, 3.0, 700)]
    prices, greeks, status = ctx.price_greeks(reqs, method=method, base_case=B)
    _check(method, reqs, prices, greeks, status)


def test_greeks_edge_cases(ctx):
    """T < 3: a price and NaN sensitivities; a bad request: NaN everywhere;
    the plain stencil method has no sensitivities (AOP_EINVAL)."""
    reqs = [wl.fixed_call(0, 2), wl.fixed_call(0, 3), wl.fixed_bsm_put(3), wl.fixed_put(aop.TRINOMIAL_PUT, 3),
            wl.Request(0, -1.0, 100.0, 0.05, 0.02, 0.2, 1.0, 100)]
    prices, greeks, status = ctx.price_greeks(reqs, method=aop.FFT_FP64)
    assert status.tolist() == [0, 0, 0, 0, 1]
    assert np.isfinite(prices[:4]).all() and np.isnan(prices[4])
    assert np.isnan(greeks[0]).all() and np.isnan(greeks[4]).all()
    _check(aop.FFT_FP64, reqs[1:4], prices[1:4], greeks[1:4], status[1:4])
    with pytest.raises(aop.AopError) as e:
        ctx.price_greeks(reqs[1:2], method=aop.STENCIL_FP64)
    assert e.value.code == 1


def test_greeks_pde_at_the_root_large_T(ctx):
    """At T = 2^16, beyond the oracle's reach in a test, the American
    sensitivities satisfy the Black-Scholes-Merton equation at the root
    (continuation region) to O(dt), and without early exercise they match
    the Black-Scholes-Merton closed forms."""
    from tests import closed_forms as cf
    T = 1 << 16
    reqs = [wl.Request(aop.BINOMIAL_PUT, 105.0, 100.0, 0.05, 0.02, 0.3, 1.0, T),
            wl.Request(aop.TRINOMIAL_PUT, 110.0, 100.0, 0.06, 0.01, 0.25, 2.0, T, math.sqrt(3)),
            wl.Request(aop.BSM_PUT, 100.0, 100.0, 0.05, 0.03, 0.3, 1.0, T),
            wl.Request(aop.BINOMIAL_CALL, 95.0, 100.0, 0.03, 0.05, 0.25, 1.5, T),
            wl.Request(aop.BINOMIAL_CALL, 95.0, 100.0, 0.03, 0.0, 0.25, 1.5, T),
            wl.Request(aop.TRINOMIAL_PUT, 95.0, 100.0, 0.0, 0.02, 0.35, 1.0, T, math.sqrt(3))]
    # the last two have whole rows red: node prices past the FP32 methods'
    # range at this T (AOP_ERANGE), so they run in FP64
    p1, g1, s1 = ctx.price_greeks(reqs[:4], method=aop.FFT_DF32)
    p2, g2, s2 = ctx.price_greeks(reqs[4:], method=aop.FFT_FP64)
    prices, greeks, status = np.concatenate([p1, p2]), np.concatenate([g1, g2]), np.concatenate([s1, s2])
    assert (status == 0).all()
    for r, v, (d, g, t) in zip(reqs, prices, greeks):
        res = t + 0.5 * r.sigma ** 2 * r.S0 ** 2 * g + (r.r - r.q) * r.S0 * d - r.r * v
        assert abs(res) <= 1e-3 * max(r.r * v, 1e-2), (r, res)
    for r, (d, g, t) in list(zip(reqs, greeks))[4:]:
        bd, bg, bt = cf.bs_greeks(r.S0, r.K, r.r, r.q, r.sigma, r.expiry, r.model == aop.BINOMIAL_CALL)
        assert abs(d - bd) < 1e-4 and abs(g - bg) < 1e-3 * bg and abs(t - bt) < 1e-3 * abs(bt), (r, d, bd, g, bg, t, bt)
