"""The allocation-free linear advance (aop_linear_advance_noalloc) against the
context-based one (aop_linear_advance_device), through the C ABI.

The allocation-free entry point serves callers that cannot allocate device
memory at call time; its scratch is a static device array shared by all calls.
This file is collected last so that a run stopping at the first failure has
already run every other test.  Two calls in a row check that the state left in
the shared array by one call does not leak into the next.
"""
import numpy as np
import pytest

import paper_2303_02317_gb300 as aop

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", [aop.FFT_FP64, aop.FFT_FP32SPLIT], ids=["fft64", "fft32"])
def test_noalloc_matches_context_entry_point(method, oracle_lib):
    """Two calls in a row: the widest segment the entry point takes, in more
    segments than it runs CTAs (40 > 16), then a short binomial one; each
    against the context entry point and the oracle's plain stencil loop."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    with aop.Context(0) as ctx:
        for call, (nw, W, h, count) in enumerate([(3, aop.NOALLOC_MAX_W, 300, 40), (2, 700, 90, 3)]):
            rng = np.random.default_rng(1000 + 17 * call + method)
            w = rng.uniform(0.2, 1.0, nw)
            w = list(w / w.sum() * 0.999)
            x = np.abs(rng.normal(size=(count, W))) * 50.0
            nout = W - (nw - 1) * h
            dx = torch.tensor(x, dtype=torch.float64, device="cuda")
            ref = torch.full((count, nout), float("nan"), dtype=torch.float64, device="cuda")
            got = torch.full((count, nout), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            ctx.linear_advance_device(method, w, count, W, h, dx.data_ptr(), ref.data_ptr())
            stream.wait_stream(torch.cuda.current_stream())
            aop.linear_advance_noalloc(method, w, count, W, h, dx.data_ptr(), got.data_ptr(),
                                       stream=stream.cuda_stream)
            stream.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.isfinite(g).all()
            scale = np.abs(x).max()
            tol = 1e-12 * scale if method == aop.FFT_FP64 else 1e-6 * scale
            assert np.abs(g - r).max() <= tol
            want = oracle_lib.linear_advance(x, w, h)
            assert np.abs(g - want).max() <= tol


def test_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    W = aop.NOALLOC_MAX_W + 1
    dx = torch.zeros((1, W), dtype=torch.float64, device="cuda")
    dy = torch.zeros((1, W), dtype=torch.float64, device="cuda")
    with pytest.raises(aop.AopError) as ei:
        aop.linear_advance_noalloc(aop.FFT_FP64, [0.5, 0.5], 1, W, 10, dx.data_ptr(), dy.data_ptr())
    assert ei.value.code == 1
