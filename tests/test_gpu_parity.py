"""GPU parity: every method against the FP64 CPU oracle, element by element
(price and the divider of every lattice row), through the C ABI."""
import math

import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import parity

pytestmark = pytest.mark.gpu

METHODS = [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.STENCIL_FP64, aop.FFT_DF32, aop.STENCIL_DF32]
MNAME = {0: "fft64", 1: "fft32", 2: "stencil", 3: "df32", 4: "stencil_df32"}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


def _check(req, method, base_case=0):
    d = req.as_dict() if hasattr(req, "as_dict") else dict(req)
    ref, bref, margin = oracle.price_american(d, with_boundary=True, with_margin=True)
    got, b = aop.price_american_ex(d, method=method, base_case=base_case, boundary=True)
    tol = parity.price_tol(method, ref, d["K"])
    assert abs(got - ref) <= tol, (MNAME[method], d, got, ref, abs(got - ref), tol)
    bad, ndiff = parity.check_boundary(method, d, b, bref, margin)
    assert not bad, (MNAME[method], d, "rows", bad[:8], [(int(b[i]), int(bref[i]), margin[i]) for i in bad[:4]])
    return got, ref, ndiff


def _edge_cases():
    base = wl.fixed_call(0, 300)
    out = [
        base.with_T(1), base.with_T(2), base.with_T(3), base.with_T(7),
        wl.fixed_call(1, 1), wl.fixed_call(1, 5), wl.fixed_bsm_put(1), wl.fixed_bsm_put(2),
        wl.fixed_bsm_put(5),
        # deep in the money with a large yield: immediate exercise, all green
        wl.Request(0, 150.0, 50.0, 0.01, 0.08, 0.15, 2.0, 257),
        wl.Request(1, 150.0, 50.0, 0.01, 0.08, 0.15, 2.0, 257, math.sqrt(3)),
        # no yield: the call is never exercised early, whole rows red
        wl.Request(0, 100.0, 100.0, 0.05, 0.0, 0.3, 1.0, 513),
        wl.Request(1, 100.0, 100.0, 0.05, 0.0, 0.3, 1.0, 513, 0.0, 1),
        # far out of the money call
        wl.Request(0, 50.0, 150.0, 0.05, 0.02, 0.2, 0.5, 300),
        # puts: no rate (no early exercise), deep in and out of the money
        wl.Request(2, 100.0, 100.0, 0.0, 0.0, 0.3, 1.0, 400),
        wl.Request(2, 100.0, 100.0, 1e-6, 0.0, 0.6, 3.0, 400),   # divider jumps at row 1
        wl.Request(2, 150.0, 50.0, 0.05, 0.0, 0.2, 1.0, 400),
        wl.Request(2, 50.0, 150.0, 0.08, 0.0, 0.2, 3.0, 400),
        # the paper's experiment parameters (Sec. 5)
        wl.paper_params(0, 1000), wl.paper_params(1, 1000), wl.paper_params(2, 1000),
        wl.single_binomial_t2048(),
    ]
    return out


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_edge_cases(ctx, method):
    for r in _edge_cases():
        _check(r, method)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_random_small(ctx, method):
    for r in wl.random_small(45, seed=11, T_range=(8, 700)):
        _check(r, method)


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.FFT_DF32], ids=["fft64", "fft32", "df32"])
@pytest.mark.parametrize("B", [2, 8, 31, 32, 47, 63, 64])
def test_base_case_heights(ctx, method, B):
    """The trapezoid cut does not change the result (any base-case height,
    powers of two or not: the recursion's heights are B times powers of two)."""
    for r in wl.random_small(9, seed=100 + B, T_range=(200, 1500)):
        _check(r, method, base_case=B)


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.FFT_DF32], ids=["fft64", "fft32", "df32"])
@pytest.mark.parametrize("B", [63, 64])
def test_wide_rows_at_the_largest_base_case(ctx, method, B):
    """Whole rows red (no yield) with the largest base case: the chain's last
    trapezoids are as wide as the lattice rows (up to 2 x 175 cells), wider
    than one base case holds, and must be cut further."""
    for T in (150, 170, 240):
        for r in (wl.Request(1, 100.0, 100.0, 0.05, 0.0, 0.3, 1.0, T, math.sqrt(3)),
                  wl.Request(1, 120.0, 100.0, 0.08, 1e-4, 0.2, 2.0, T, 0.0, 1),
                  wl.Request(0, 100.0, 100.0, 0.05, 0.0, 0.3, 1.0, T),
                  wl.Request(2, 100.0, 100.0, 0.05, 0.0, 0.3, 1.0, T)):
            _check(r, method, base_case=B)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
@pytest.mark.parametrize("T", [4095, 8192])
def test_configs_mid_size(ctx, method, T):
    """Benchmark parameter sets at sizes the oracle runs in seconds: several
    shared-memory tiles, multi-pass transforms and ragged tails."""
    for r in (wl.fixed_call(0, T), wl.fixed_call(1, T), wl.fixed_call(1, T, wl.TRI_PAPER),
              wl.fixed_bsm_put(T)):
        _check(r, method)


_ORACLE_2_16 = {}


def _oracle_full(req):
    """Oracle price, dividers and margins on all host cores, once per request."""
    key = tuple(sorted(req.items()))
    if key not in _ORACLE_2_16:
        _ORACLE_2_16[key] = oracle.price_american(req, nthreads=0, with_boundary=True, with_margin=True)
    return _ORACLE_2_16[key]


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_configs_at_2_16(ctx, method):
    """The benchmark's fixed-parameter sets at T = 2^16, the largest size at
    which the oracle is the reference: binomial, trinomial (Boyle and the
    paper's form) and the BSM put; price and every row's divider."""
    T = 1 << 16
    for r in (wl.fixed_call(0, T), wl.fixed_call(1, T), wl.fixed_call(1, T, wl.TRI_PAPER), wl.fixed_bsm_put(T)):
        d = r.as_dict()
        ref, bref, margin = _oracle_full(d)
        got, b = aop.price_american_ex(d, method=method, boundary=True)
        tol = parity.price_tol(method, ref, d["K"])
        assert abs(got - ref) <= tol, (MNAME[method], d, got, ref, abs(got - ref), tol)
        bad, _ = parity.check_boundary(method, d, b, bref, margin)
        assert not bad, (MNAME[method], d, "rows", bad[:8])


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_extreme_parameters(ctx, method):
    """Corners of the benchmark parameter box at T = 8192: the widest lattices
    (sigma = 0.6, three years, node prices near e^{+-200}) and the most skewed
    probabilities (sigma = 0.1, r = 0.08)."""
    T = 8192
    cases = [
        wl.Request(0, 150.0, 50.0, 0.08, 0.005, 0.6, 3.0, T),
        wl.Request(1, 150.0, 50.0, 0.08, 0.005, 0.6, 3.0, T, math.sqrt(3)),
        wl.Request(1, 50.0, 150.0, 0.0, 0.06, 0.6, 3.0, T, math.sqrt(3)),
        wl.Request(0, 100.0, 100.0, 0.08, 0.005, 0.1, 0.1, T),
        wl.Request(1, 100.0, 100.0, 0.08, 0.005, 0.1, 3.0, T, 0.0, 1),
        wl.Request(2, 50.0, 150.0, 0.08, 0.0, 0.6, 3.0, T),
        wl.Request(2, 150.0, 50.0, 0.08, 0.0, 0.1, 3.0, T),
        wl.Request(2, 100.0, 100.0, 0.001, 0.0, 0.6, 0.1, T),
    ]
    for r in cases:
        _check(r, method)


def test_fp32_range_status(ctx):
    """No yield, three years at sigma 0.6 and T = 8192: every row is red and the
    deep in-the-money values reach e^94 S0.  The FP32 D&C methods answer
    AOP_ERANGE (8) for that option only; FP64 prices it, and so does the
    doubled-FP32 stencil, whose clamp of the exercise values at 1e30 lies 64
    log-units from the money, out of the walk's reach."""
    wide = wl.Request(0, 100.0, 100.0, 0.05, 0.0, 0.6, 3.0, 8192)
    fine = wl.fixed_call(0, 8192)
    ref = oracle.price_american(wide.as_dict())
    prices, status = ctx.price_batch([wide, fine], method=aop.STENCIL_DF32)
    assert (status == 0).all()
    assert abs(prices[0] - ref) <= parity.price_tol(aop.STENCIL_DF32, ref, wide.K), (prices[0], ref)
    for m in (aop.FFT_FP32SPLIT, aop.FFT_DF32):
        prices, status = ctx.price_batch([wide, fine], method=m)
        assert status[0] == 8 and np.isnan(prices[0]), (m, status, prices)
        assert status[1] == 0
    got = aop.price_american_ex(wide.as_dict(), method=aop.FFT_FP64)
    assert abs(got - ref) <= parity.price_tol(aop.FFT_FP64, ref, wide.K)


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.FFT_DF32], ids=["fft64", "fft32", "df32"])
def test_lattice_beyond_fp64_range(ctx, method):
    """A trinomial lattice whose extreme node prices pass e^709 (sigma 0.58,
    2.9 years, T = 174130): plain backward induction overflows there, while
    the D&C leaves the cells beyond the FP64 range green (they lie far above
    the exercise boundary).  Checked against the same option at T = 120000
    (node prices within range, plain FP64 stencil): lattice convergence
    O(1/T) bounds the difference by 1e-3 of the price; the methods agree with
    the FP64 D&C within their tolerances."""
    args = (108.40797915083324, 60.46799288988718, 0.009004600663437846, 0.016617322323111118,
            0.5817829465682484, 2.924264468806686)
    r = wl.Request(1, *args, 174130, math.sqrt(3))
    r_in = wl.Request(1, *args, 120000, math.sqrt(3))
    got, st = ctx.price_batch([r], method=method)
    p64, st64 = ctx.price_batch([r], method=aop.FFT_FP64)
    ref, sst = ctx.price_batch([r_in], method=aop.STENCIL_FP64)
    assert st[0] == 0 and st64[0] == 0 and sst[0] == 0 and np.isfinite(ref[0])
    assert abs(p64[0] - ref[0]) <= 1e-3 * ref[0], (p64, ref)
    assert abs(got[0] - p64[0]) <= parity.price_tol(method, p64[0], r.K), (got, p64)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_batch_matches_single(ctx, method):
    reqs = wl.random_small(24, seed=5, T_range=(16, 900))
    prices, status = ctx.price_batch(reqs, method=method)
    assert (status == 0).all()
    for r, p in zip(reqs, prices):
        ref = oracle.price_american(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(method, ref, r.K)


def test_invalid_and_unstable_requests(ctx):
    good = wl.fixed_call(0, 64)
    bad = [
        wl.Request(0, 0.0, 100, 0.05, 0.03, 0.2, 1.0, 64),      # S0 <= 0
        wl.Request(0, 100, 100, 0.05, 0.03, 0.0, 1.0, 64),      # sigma <= 0
        wl.Request(5, 100, 100, 0.05, 0.01, 0.2, 1.0, 64),      # unknown model
        wl.Request(0, 100, 100, 0.5, 0.0, 0.001, 1.0, 4),       # p > 1
    ]
    for method in METHODS:
        prices, status = ctx.price_batch([good] + bad + [good], method=method)
        assert status.tolist() == [0, 1, 1, 1, 2, 0]
        assert np.isnan(prices[1:5]).all()
        ref = oracle.price_american(good.as_dict())
        assert abs(prices[0] - ref) <= parity.price_tol(method, ref, good.K)
        assert prices[0] == prices[-1]


@pytest.mark.parametrize("method", [aop.FFT_DF32, aop.FFT_FP32SPLIT])
def test_walker_placement_bit_equal(ctx, method):
    """Which warp of a CTA walks the recursion (all walkers of an SM on one
    sub-partition, or spread over them) changes the schedule, not the
    arithmetic: prices are bit-equal, and equal the oracle within tolerance."""
    reqs = wl.random_small(24, seed=41, T_range=(200, 3000))
    p0, s0 = ctx.price_batch(reqs, method=method)
    p1, s1 = ctx.price_batch(reqs, method=method, flags=aop.FLAG_SPREAD_WALKERS)
    assert (s0 == 0).all() and (s1 == 0).all()
    assert np.array_equal(p0, p1)
    for r, p in zip(reqs, p1):
        ref = oracle.price_american(r.as_dict())
        assert abs(p - ref) <= parity.price_tol(method, ref, r.K), (r, p, ref)
