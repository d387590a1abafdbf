"""Serving sessions (continuous pricing through one persistent kernel): each
result equals the same request priced alone in a batch, requests that arrive
while others are in flight are admitted, an idle kernel is relaunched, and bad
requests come back with their status.  Through the C ABI (aop_server_*)."""
import time

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


def _stream(n, seed, mean_gap_s, T_range):
    reqs = wl.random_small(n, seed=seed, T_range=T_range)
    rng = np.random.default_rng(seed + 1)
    gaps = rng.exponential(mean_gap_s, n)
    return reqs, np.cumsum(gaps) - gaps[0]


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.FFT_DF32], ids=["fft64", "fft32", "df32"])
def test_stream_matches_alone(ctx, method):
    """Each price of a mixed stream (binomial, trinomial, BSM; T from 64 to
    2000; arrivals every 0.2 ms on average, so many overlap on the device)
    equals the price of the same request alone, bit for bit."""
    reqs, arrivals = _stream(48, 21, 2e-4, (64, 2000))
    with aop.Server(ctx, capacity=64, T_max=2048, method=method, base_case=16) as srv:
        info = srv.info()
        assert info["slots"] >= 1
        prices, status, lat = srv.serve_stream(reqs, arrivals, timeout_s=120.0)
    assert (status == 0).all(), status
    assert (lat > 0).all()
    alone = np.array([ctx.price_batch([r], method=method, base_case=16)[0][0] for r in reqs])
    assert np.array_equal(prices, alone), np.max(np.abs(prices - alone))
    for r, p in list(zip(reqs, prices))[:8]:
        ref = oracle.price_american(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(method, ref, r.K), (r, p, ref)


@pytest.mark.parametrize("method", [aop.FFT_DF32, aop.FFT_FP32SPLIT], ids=["df32", "fft32"])
def test_freed_slots_take_new_requests(method):
    """A workspace cap that holds four options at T = 2^13 and 96 requests
    arriving faster than four slots price them: requests wait for a slot and
    are admitted into slots as they free.  Every price equals the same
    request priced alone, bit for bit."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    T_max = 1 << 13
    cap = aop.workspace_bytes(method, T_max, 4, base_case=31)
    reqs, arrivals = _stream(96, 41, 5e-5, (200, T_max))
    with aop.Context(0, workspace_cap_bytes=cap) as c:
        with aop.Server(c, capacity=96, T_max=T_max, method=method, base_case=31) as srv:
            assert 1 <= srv.info()["slots"] <= 4
            prices, status, lat = srv.serve_stream(reqs, arrivals, timeout_s=300.0)
        assert (status == 0).all(), status
        alone = np.array([c.price_batch([r], method=method, base_case=31)[0][0] for r in reqs])
    assert np.array_equal(prices, alone), np.max(np.abs(prices - alone))
    # at some arrival more requests were outstanding than there are slots, so
    # some waited and were admitted into a slot freed by another
    done = arrivals + lat
    outstanding = max(int(np.sum((arrivals <= t) & (done > t))) for t in arrivals)
    assert outstanding > 4, outstanding


def test_submit_poll_and_idle_relaunch(ctx):
    """Requests submitted one at a time are priced; after more than the
    kernel's 2 s idle limit the next request relaunches it."""
    reqs = wl.random_small(4, seed=33, T_range=(100, 400))
    with aop.Server(ctx, capacity=8, T_max=512, method=aop.FFT_DF32) as srv:
        ids = [srv.submit(r) for r in reqs[:2]]
        got = {}
        t0 = time.time()
        while len(got) < 2 and time.time() - t0 < 60:
            for i in ids:
                done, p, st = srv.poll(i)
                if done:
                    got[i] = (p, st)
        assert len(got) == 2
        time.sleep(2.6)                      # the kernel has exited by now
        ids2 = [srv.submit(r) for r in reqs[2:]]
        t0 = time.time()
        while len(got) < 4 and time.time() - t0 < 60:
            for i in ids2:
                done, p, st = srv.poll(i)
                if done:
                    got[i] = (p, st)
        assert len(got) == 4
    for i, r in enumerate(reqs):
        p, st = got[i]
        assert st == 0
        ref = oracle.price_american(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(aop.FFT_DF32, ref, r.K)


def test_bad_requests_and_busy_context(ctx):
    good = wl.fixed_call(0, 200)
    too_long = wl.fixed_call(1, 600)              # above the session's T_max
    bad = wl.Request(0, -1.0, 100.0, 0.05, 0.02, 0.2, 1.0, 100)
    with aop.Server(ctx, capacity=4, T_max=256, method=aop.FFT_FP64) as srv:
        with pytest.raises(aop.AopError) as e:
            ctx.price_batch([good], method=aop.FFT_FP64)
        assert e.value.code == 6                  # AOP_EBUSY while the session holds the workspace
        prices, status, _ = srv.serve_stream([good, too_long, bad], [0.0, 0.0, 0.0], timeout_s=60.0)
        assert status[0] == 0 and status[1] == 1 and status[2] == 1
        assert np.isnan(prices[1]) and np.isnan(prices[2])
        with pytest.raises(aop.AopError):
            srv.serve_stream([good, good], [0.0, 0.0])    # capacity 4: 3 used
    ref = oracle.price_american(good.as_dict())
    assert abs(prices[0] - ref) <= parity.price_tol(aop.FFT_FP64, ref, good.K)
    # the context serves batches again once the session is closed
    p, s = ctx.price_batch([good], method=aop.FFT_FP64)
    assert s[0] == 0 and p[0] == prices[0]
