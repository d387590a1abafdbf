"""GPU parity of the FFT linear advance (the linear-stencil step inside every
trapezoid) against the oracle's plain definition: the stencil applied h times
in FP64 (oracle.linear_advance, pinned to the binomial and trinomial
coefficients on the CPU)."""
import numpy as np
import pytest

import oracle
import paper_2303_02317_gb300 as aop

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = aop.Context(0)
    yield c
    c.close()


CASES = [
    # (nw, W, h, count)
    (2, 5, 1, 3), (2, 64, 31, 2), (2, 100, 37, 4), (3, 100, 10, 2), (3, 4096, 1000, 2),
    (2, 4097, 2000, 1), (3, 5000, 1200, 2), (2, 70000, 3000, 1), (3, 65537, 8000, 1),
    # around the tile sizes of the real-input transforms (16-byte values: N/2
    # complex points in one 2^11 tile up to N = 2^12, mirror blocks beyond)
    (2, 2048, 3, 2), (3, 2049, 5, 1), (2, 8192, 100, 1), (3, 16385, 2000, 1),
]


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT, aop.FFT_DF32], ids=["fft64", "fft32", "df32"])
@pytest.mark.parametrize("nw,W,h,count", CASES)
def test_linear_advance(ctx, method, nw, W, h, count):
    rng = np.random.default_rng(W * 7 + h)
    w = rng.uniform(0.2, 1.0, nw)
    w = w / w.sum() * 0.999
    x = np.abs(rng.normal(size=(count, W))) * rng.uniform(0.1, 100.0)
    ref = oracle.linear_advance(x, w, h)
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    nout = W - (nw - 1) * h
    dy = torch.full((count, nout), float("nan"), dtype=torch.float64, device="cuda")
    ctx.linear_advance_device(method, list(w), count, W, h, dx.data_ptr(), dy.data_ptr())
    got = dy.cpu().numpy()
    # rounding relative to the segment's largest value: FP64 and doubled FP32
    # (~2^-48 a stage, summed over up to 2^17 points) below 5e-11, the FP32
    # split at the FP32 level
    scale = np.abs(x).max()
    tol = {aop.FFT_FP64: 1e-12, aop.FFT_DF32: 5e-11, aop.FFT_FP32SPLIT: 1e-6}[method] * scale
    err = np.abs(got - ref).max()
    assert err <= tol, (err, tol, err / scale)
