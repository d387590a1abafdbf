"""Schedules of the divide-and-conquer pricer (base-case height, options per
SM, transform tile, transform radix): every schedule prices within the parity
tolerance of the oracle, and the autotuner keeps its picks per context by
method, size and model class.  Through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
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


CASES = [wl.fixed_call(0, 6000), wl.fixed_call(1, 3000), wl.fixed_call(1, 3001, wl.TRI_PAPER),
         wl.fixed_bsm_put(3000), wl.Request(0, 80.0, 100.0, 0.06, 0.02, 0.4, 2.0, 4097)]


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_DF32, aop.FFT_FP32SPLIT], ids=["fft64", "df32", "fft32"])
@pytest.mark.parametrize("lg_tile,radix", [(9, 4), (9, 2), (10, 2), (11, 4)])
def test_transform_schedules_match_oracle(ctx, method, lg_tile, radix):
    """Rows of 6000-12000 cells take multi-pass transforms with a 2^9 tile and
    single-tile ones with 2^11; radix-2 stages replace the radix-4 steps.  The
    prices stay within the method's parity tolerance of the oracle."""
    prices, status = ctx.price_batch(CASES, method=method, base_case=63, lg_tile=lg_tile, radix=radix)
    assert (status == 0).all(), status
    for r, p in zip(CASES, prices):
        ref = oracle.price_american(r.as_dict(), nthreads=0)
        assert abs(p - ref) <= parity.price_tol(method, ref, r.K), (r, lg_tile, radix, p, ref)


def test_autotune_keeps_picks_per_size_and_model():
    """Two tunings on one context (binomial calls at T = 2048, trinomial calls
    at T = 4096) are both kept: a batch of each kind gets its own pick, a
    mixed batch of another size the pick of the nearest size, and explicit
    options override the picks.  Prices with the picks match the oracle."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bino = wl.random_small(6, seed=71, T_range=(1500, 2048), models=(0,))
    trin = wl.random_small(6, seed=72, T_range=(3000, 4096), models=(1,))
    with aop.Context(0) as c:
        assert c.schedule(bino, aop.FFT_DF32)["lg_tile"] == 10            # library defaults before tuning
        pb = c.autotune(bino, aop.FFT_DF32)
        pt = c.autotune(trin, aop.FFT_DF32)
        for p in (pb, pt):
            assert p["base_case"] in (16, 31, 32, 47, 63, 64) and p["ctas_per_sm"] in (1, 2, 3, 4)
            assert p["lg_tile"] in (9, 10, 11) and p["radix"] in (2, 4)
        assert c.schedule(bino, aop.FFT_DF32) == pb
        assert c.schedule(trin, aop.FFT_DF32) == pt
        near = wl.random_small(4, seed=73, T_range=(3500, 4000), models=(0, 1))
        assert c.schedule(near, aop.FFT_DF32) == pt                       # nearest size bucket
        assert c.schedule(bino, aop.FFT_FP64)["lg_tile"] == 10            # per method
        prices, status = c.price_batch(trin, method=aop.FFT_DF32)
        assert (status == 0).all()
        for r, p in zip(trin, prices):
            ref = oracle.price_american(r.as_dict(), nthreads=0)
            assert abs(p - ref) <= parity.price_tol(aop.FFT_DF32, ref, r.K)
