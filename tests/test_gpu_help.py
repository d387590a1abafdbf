"""Helping (on by default for D&C batches; AOP_FLAG_NO_HELP turns it off),
through the C ABI.

An option's multi-pass linear advances go on its CTA's board in global
memory, where its own workers and the workers of idle CTAs take them (Sec.
2.3: the advances of a trapezoid run beside the recursion next to it).  The
arithmetic of an advance does not depend on which SM or how many warps run it,
so prices and dividers are bit-equal to a launch without helping.  These tests
check that, check that helpers did run advances, and check the failure path
(no worker takes a task) with helping on.
"""
import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import parity

pytestmark = pytest.mark.gpu

OFF = aop.FLAG_NO_HELP


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


# single options whose rows need transforms of 2^12 .. 2^16 points (multi-pass
# at the default 2^10-value tile)
SINGLES = [wl.fixed_call(0, 1 << 14), wl.fixed_call(1, 1 << 13), wl.fixed_call(1, 6001, wl.TRI_PAPER),
           wl.fixed_bsm_put(1 << 13), wl.fixed_put(0, 5000), wl.fixed_put(1, 3000),
           wl.Request(0, 80.0, 100.0, 0.06, 0.02, 0.4, 2.0, 20000)]
METHODS = [aop.FFT_FP64, aop.FFT_DF32, aop.FFT_FP32SPLIT]
IDS = ["fft64", "df32", "fft32"]


@pytest.mark.parametrize("method", METHODS, ids=IDS)
def test_single_options_bit_equal(ctx, method):
    """One option per launch with three helper CTAs: the same price, bit for
    bit, as without helping; the helpers ran some of its advances (none in the
    FP32-split mode, which does not help)."""
    helped = 0
    for r in SINGLES:
        # the same height both ways (untuned, a helped trinomial takes 31)
        p0, s0 = ctx.price_batch([r], method=method, base_case=63, flags=OFF)
        p1, s1 = ctx.price_batch([r], method=method, base_case=63)
        helped += ctx.stats()["helped_advances"]
        assert s0[0] == 0 and s1[0] == 0, (r, s0, s1)
        assert p1[0] == p0[0], (r, p0[0], p1[0])
    assert (helped == 0) if method == aop.FFT_FP32SPLIT else (helped > 0)


def test_single_dividers_bit_equal(ctx):
    """Every row's divider is the same with helping, and the price is within
    the parity tolerance of the oracle."""
    for r in SINGLES[:4]:
        d = r.as_dict()
        p0, b0 = aop.price_american_ex(d, method=aop.FFT_DF32, base_case=63, boundary=True, flags=OFF)
        p1, b1 = aop.price_american_ex(d, method=aop.FFT_DF32, base_case=63, boundary=True)
        assert p1 == p0
        assert np.array_equal(b0, b1)
    r = SINGLES[1]
    ref = oracle.price_american(r.as_dict(), nthreads=0)
    p, _ = ctx.price_batch([r], method=aop.FFT_DF32)
    assert abs(p[0] - ref) <= parity.price_tol(aop.FFT_DF32, ref, r.K)


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("method", [aop.FFT_DF32, aop.FFT_FP64], ids=["df32", "fft64"])
def test_small_batch_bit_equal(ctx, method):
    """A batch of a quarter as many options as SMs, of mixed sizes and models:
    three helping CTAs per option, and CTAs whose options finish early help
    the rest.  Every price is bit-equal to the launch without helping, and a
    second launch on the same workspace (whose boards, left by the last
    launch, must be skipped) gives the same prices again."""
    rng = np.random.default_rng(2303)
    reqs = wl.random_small(_sms() // 4, seed=7, T_range=(1500, 12000), models=(0, 1, 2))
    p0, s0 = ctx.price_batch(reqs, method=method, flags=OFF)
    p1, s1 = ctx.price_batch(reqs, method=method)
    st = ctx.stats()
    assert (s0 == 0).all() and (s1 == 0).all()
    assert np.array_equal(p0, p1), np.nonzero(p0 != p1)[0][:8]
    assert st["helped_advances"] > 0
    order = rng.permutation(len(reqs))
    p2, s2 = ctx.price_batch([reqs[i] for i in order], method=method)
    assert (s2 == 0).all()
    assert np.array_equal(p2, p0[order])


def test_large_batch_does_not_help(ctx):
    """More options than SMs: no helping CTA (they would share SMs with the
    options' recursions), the same prices."""
    reqs = wl.random_small(_sms() + 10, seed=8, T_range=(1500, 6000), models=(0, 1, 2))
    p0, s0 = ctx.price_batch(reqs, method=aop.FFT_DF32, flags=OFF)
    p1, s1 = ctx.price_batch(reqs, method=aop.FFT_DF32)
    assert (s0 == 0).all() and (s1 == 0).all() and np.array_equal(p0, p1)
    assert ctx.stats()["helped_advances"] == 0


def test_stall_with_helping_times_out_and_recovers(ctx):
    """No worker, own or helping, takes a task: each option ends with
    AOP_ETIMEOUT and a NaN price, the helpers stop, and the next call prices
    normally."""
    reqs = [wl.fixed_call(0, 4096), wl.fixed_bsm_put(4096)]
    prices, status = ctx.price_batch(reqs, method=aop.FFT_DF32, flags=aop.FLAG_TEST_STALL)
    assert (status == 5).all() and np.isnan(prices).all(), (status, prices)
    p0, s0 = ctx.price_batch(reqs, method=aop.FFT_DF32, flags=OFF)
    p1, s1 = ctx.price_batch(reqs, method=aop.FFT_DF32)
    assert (s0 == 0).all() and (s1 == 0).all() and np.array_equal(p0, p1)


def test_small_three_point_batches_default_to_height_31():
    """Untuned, a batch of three-point lattices only that is small enough to
    help takes base case 31 (the spare SMs absorb the extra advances); a
    binomial batch, a large batch and the FP32-split method keep 63."""
    c = aop.Context(0)
    try:
        tri = [wl.fixed_call(1, 1 << 13)]
        assert c.schedule(tri, aop.FFT_DF32)["base_case"] == 31
        assert c.schedule(tri, aop.FFT_FP32SPLIT)["base_case"] == 63
        assert c.schedule([wl.fixed_call(0, 1 << 13)], aop.FFT_DF32)["base_case"] == 63
        assert c.schedule(tri * _sms(), aop.FFT_DF32)["base_case"] == 63
        p, s = c.price_batch(tri, method=aop.FFT_DF32)
        ref = oracle.price_american(tri[0].as_dict(), nthreads=0)
        assert s[0] == 0 and abs(p[0] - ref) <= parity.price_tol(aop.FFT_DF32, ref, tri[0].K)
    finally:
        c.close()
