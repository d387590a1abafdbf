"""GPU parity of the put variants against the FP64 CPU oracle, through the C
ABI: binomial and trinomial American puts (priced by the library as the call
of the mirrored lattice; the oracle runs the put recursion itself) and the BSM
put with a dividend yield.  Prices within the method's tolerance and the
divider of every row equal outside the tie band, as for the calls."""
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
BP, TP = aop.BINOMIAL_PUT, aop.TRINOMIAL_PUT


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
    tol = parity.price_tol(method, ref, max(d["K"], d["S0"]))
    assert abs(got - ref) <= tol, (MNAME[method], d, got, ref, abs(got - ref), tol)
    bad, _ = parity.check_boundary(method, d, b, bref, margin)
    assert not bad, (MNAME[method], d, "rows", bad[:8], [(int(b[i]), int(bref[i]), margin[i]) for i in bad[:4]])
    return got, ref


def _edge_puts():
    S3 = math.sqrt(3)
    out = []
    for m, lam in ((BP, 0.0), (TP, S3)):
        base = wl.fixed_put(m, 300)
        out += [base.with_T(1), base.with_T(2), base.with_T(3), base.with_T(7)]
        out += [
            # deep in the money, high rate: immediate exercise on most of the lattice
            wl.Request(m, 50.0, 150.0, 0.08, 0.0, 0.15, 2.0, 257, lam),
            # no rate: never exercised early (every row without green cells)
            wl.Request(m, 100.0, 100.0, 0.0, 0.03, 0.3, 1.0, 513, lam),
            # far out of the money
            wl.Request(m, 150.0, 50.0, 0.05, 0.02, 0.2, 0.5, 300, lam),
            # yield above the rate
            wl.Request(m, 95.0, 100.0, 0.01, 0.07, 0.4, 2.5, 400, lam),
        ]
    out += [wl.fixed_put(TP, 301, wl.TRI_PAPER), wl.Request(TP, 80.0, 100.0, 0.06, 0.01, 0.25, 1.5, 333, 0.0, wl.TRI_PAPER)]
    # BSM put with a yield: ordinary, no rate, deep in and out of the money
    out += [
        wl.Request(2, 100.0, 100.0, 0.05, 0.03, 0.3, 1.0, 400),
        wl.Request(2, 100.0, 100.0, 0.0, 0.04, 0.3, 1.0, 400),
        wl.Request(2, 50.0, 150.0, 0.08, 0.02, 0.2, 3.0, 400),
        wl.Request(2, 150.0, 50.0, 0.05, 0.06, 0.2, 1.0, 400),
    ]
    return out


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_put_edge_cases(ctx, method):
    for r in _edge_puts():
        _check(r, method)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_lattice_puts_random(ctx, method):
    for r in wl.random_small(40, seed=31, T_range=(8, 700), models=(BP, TP)):
        _check(r, method)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_bsm_put_with_yield_random(ctx, method):
    for r in wl.random_small(20, seed=37, T_range=(8, 700), models=(2,), bsm_yield=True):
        _check(r, method)


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.FFT_DF32], ids=["fft64", "fft32", "df32"])
@pytest.mark.parametrize("B", [2, 16, 31, 63, 64])
def test_put_base_case_heights(ctx, method, B):
    for r in wl.random_small(9, seed=41 + B, T_range=(100, 1500), models=(BP, TP, 2), bsm_yield=True):
        _check(r, method, base_case=B)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_puts_mid_size(ctx, method):
    """T = 6000: several levels of the recursion and multi-tile transforms."""
    for r in (wl.fixed_put(BP, 6000), wl.fixed_put(TP, 6000),
              wl.Request(2, 100.0, 100.0, 0.05, 0.03, 0.3, 1.0, 6000)):
        _check(r, method)


@pytest.mark.parametrize("method", METHODS, ids=[MNAME[m] for m in METHODS])
def test_put_batch_with_boundaries_on_device(ctx, method):
    """The device batch entry point returns the put dividers in the put's own
    columns (the mirror pass), next to calls and BSM puts in the same batch."""
    torch = pytest.importorskip("torch")
    reqs = wl.random_small(12, seed=43, T_range=(30, 500), models=(BP, 0, TP, 1, 2), bsm_yield=True)
    arr = aop.requests_array(reqs)
    dev = torch.device("cuda:0")
    d_reqs = torch.from_numpy(arr.view(np.uint8).copy()).to(dev)
    n = len(reqs)
    offs = np.concatenate([[0], np.cumsum([r.T + 1 for r in reqs])[:-1]]).astype(np.int64)
    d_off = torch.from_numpy(offs).to(dev)
    d_b = torch.full((int(sum(r.T + 1 for r in reqs)),), -7, dtype=torch.int32, device=dev)
    d_p = torch.empty(n, dtype=torch.float64, device=dev)
    d_s = torch.empty(n, dtype=torch.int32, device=dev)
    ctx.price_batch_device(n, d_reqs.data_ptr(), d_p.data_ptr(), d_s.data_ptr(), d_b.data_ptr(),
                           d_off.data_ptr(), method=method)
    torch.cuda.synchronize()
    p, s, b = d_p.cpu().numpy(), d_s.cpu().numpy(), d_b.cpu().numpy()
    assert (s == 0).all(), s
    for i, r in enumerate(reqs):
        d = r.as_dict()
        ref, bref, margin = oracle.price_american(d, with_boundary=True, with_margin=True)
        assert abs(p[i] - ref) <= parity.price_tol(method, ref, max(r.K, r.S0)), (r, p[i], ref)
        bi = b[offs[i]: offs[i] + r.T + 1]
        bad, _ = parity.check_boundary(method, d, bi, bref, margin)
        assert not bad, (MNAME[method], r, bad[:8])


def test_european_puts(ctx):
    """European puts by one FFT advance: the lattice sums and the BSM scheme
    without the max, against the oracle's European lattice."""
    reqs = wl.random_small(12, seed=47, T_range=(50, 3000), models=(BP, TP, 2), bsm_yield=True)
    prices, status = ctx.price_european(reqs)
    assert (status == 0).all()
    for r, p in zip(reqs, prices):
        ref = oracle.price_european(r.as_dict())
        assert abs(p - ref) <= 1e-10 * abs(ref) + 1e-12 * max(r.K, r.S0), (r, p, ref)
