"""Failure paths on the GPU without a fault: a device wait that nothing
satisfies gives up with AOP_ETIMEOUT and leaves the context usable, and the
workspace cap bounds the options in flight (AOP_ENOMEM below one option)."""
import time

import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import parity

pytestmark = pytest.mark.gpu

AOP_ENOMEM, AOP_ETIMEOUT = 3, 5


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_DF32], ids=["fft64", "df32"])
def test_bounded_wait_gives_up_and_context_stays_usable(ctx, method):
    """With AOP_FLAG_TEST_STALL no worker takes the walker's first advance: its
    wait runs out after 20 ms and every option reports AOP_ETIMEOUT with a NaN
    price; the next call on the same context prices normally."""
    reqs = [wl.fixed_call(0, 4096), wl.fixed_call(1, 2048), wl.fixed_bsm_put(3000)]
    t0 = time.perf_counter()
    prices, status = ctx.price_batch(reqs, method=method, flags=aop.FLAG_TEST_STALL)
    assert time.perf_counter() - t0 < 20.0
    assert (status == AOP_ETIMEOUT).all(), status
    assert np.isnan(prices).all()
    prices, status = ctx.price_batch(reqs, method=method)
    assert (status == 0).all()
    for r, p in zip(reqs, prices):
        ref = oracle.price_american(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(method, ref, r.K)


def test_workspace_cap_bounds_options_in_flight():
    """A context whose workspace cap holds a few options prices a larger batch
    with fewer CTAs in flight (same prices); a cap below one option's
    workspace gives AOP_ENOMEM for the batch."""
    reqs = wl.random_small(12, seed=71, T_range=(1000, 4000))
    with aop.Context(0) as free:
        want, st = free.price_batch(reqs, method=aop.FFT_DF32)
        assert (st == 0).all()
    with aop.Context(0, workspace_cap_bytes=12 << 20) as capped:      # about four options
        got, st = capped.price_batch(reqs, method=aop.FFT_DF32)
        assert (st == 0).all()
        assert np.array_equal(got, want)
    with aop.Context(0, workspace_cap_bytes=1 << 20) as tiny:
        with pytest.raises(aop.AopError) as e:
            tiny.price_batch(reqs, method=aop.FFT_DF32)
        assert e.value.code == AOP_ENOMEM
