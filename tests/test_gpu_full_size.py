"""Parity at the benchmark's full sizes, through the C ABI.

* The precision-sweep book (256 binomial + 256 trinomial calls at T = 2^17)
  priced in one batch, as the bench times it: sampled options against the
  oracle on all host cores, price and every row's divider.
* The BSM put of configuration C3 at T = 2^18 against the plain FP64 stencil
  (the oracle-matched reference above T = 2^16): price and every row's
  divider.
"""
import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import workloads as wl
from tests import parity

pytestmark = pytest.mark.gpu

SAMPLE = (0, 256)        # a binomial and a trinomial option of the book


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aop.load()
    c = aop.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def book_oracle():
    book = wl.precision_sweep(T=1 << 17, n_binomial=256, n_trinomial=256)
    out = {}
    for i in SAMPLE:
        out[i] = oracle.price_american(book[i].as_dict(), nthreads=0, with_boundary=True, with_margin=True)
    return book, out


@pytest.mark.parametrize("method", [aop.FFT_DF32, aop.FFT_FP64], ids=["df32", "fft64"])
def test_book_in_one_batch_matches_oracle(ctx, book_oracle, method):
    """The whole book in one launch: the sampled prices within the parity
    tolerance of the oracle, every other price finite and between the
    intrinsic value and S0."""
    book, ref = book_oracle
    prices, status = ctx.price_batch(book, method=method)
    assert (status == 0).all(), np.unique(status)
    for i in SAMPLE:
        r = book[i]
        want = ref[i][0]
        assert abs(prices[i] - want) <= parity.price_tol(method, want, r.K), (i, prices[i], want)
    S = np.array([r.S0 for r in book])
    K = np.array([r.K for r in book])
    assert np.isfinite(prices).all()
    assert (prices >= np.maximum(S - K, 0.0) - 1e-9 * K).all() and (prices <= S + 1e-9).all()


def test_book_dividers_match_oracle(ctx, book_oracle):
    """Every row's divider of the sampled book options (doubled FP32, priced
    one at a time with boundary output) equals the oracle's outside its tie
    band."""
    book, ref = book_oracle
    for i in SAMPLE:
        d = book[i].as_dict()
        got, b = aop.price_american_ex(d, method=aop.FFT_DF32, boundary=True)
        want, bref, margin = ref[i]
        assert abs(got - want) <= parity.price_tol(aop.FFT_DF32, want, d["K"])
        bad, _ = parity.check_boundary(aop.FFT_DF32, d, b, bref, margin)
        assert not bad, (i, bad[:8])


def test_bsm_put_2_18_matches_fp64_stencil(ctx):
    """C3 at T = 2^18: the doubled-FP32 and FP64 D&C prices within the FP64
    tolerance of the plain FP64 stencil, and their dividers equal to the
    stencil's except where the two disagree by one cell (ties the stencil
    cannot report a margin for are rare at this size)."""
    r = wl.fixed_bsm_put(1 << 18)
    d = r.as_dict()
    ref, bref = aop.price_american_ex(d, method=aop.STENCIL_FP64, boundary=True)
    for method in (aop.FFT_DF32, aop.FFT_FP64):
        got, b = aop.price_american_ex(d, method=method, boundary=True)
        assert abs(got - ref) <= parity.price_tol(aop.FFT_FP64, ref, d["K"]), (method, got, ref)
        b, bref_ = np.asarray(b), np.asarray(bref)
        diff = np.nonzero(b != bref_)[0]
        assert len(diff) <= 16, (method, len(diff), diff[:8])
        assert (np.abs(b[diff].astype(np.int64) - bref_[diff].astype(np.int64)) <= 1).all()
