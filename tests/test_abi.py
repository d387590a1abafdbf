"""The C-ABI library builds, loads and exports every symbol its header
declares (no GPU needed; no compute call is made)."""
import ctypes
import os

import numpy as np
import pytest

import paper_2303_02317_gb300 as aop
from paper_2303_02317_gb300 import build as libbuild


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(aop.LIB_PATH):
        libbuild.build()
    return aop.load()


def test_every_declared_symbol_is_exported(lib):
    names = aop.declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_request_layout_matches_header(lib):
    assert aop.REQUEST_DTYPE.itemsize == 72
    arr = aop.requests_array([dict(model=1, S0=1.0, K=2.0, r=0.1, q=0.2, sigma=0.3, expiry=0.4,
                                   T=5, lam=1.7, tri_form=1)])
    raw = arr.tobytes()
    assert np.frombuffer(raw[0:8], dtype="<i4").tolist() == [1, 1]
    assert np.frombuffer(raw[8:56], dtype="<f8").tolist() == [1.0, 2.0, 0.1, 0.2, 0.3, 0.4]
    assert np.frombuffer(raw[56:64], dtype="<i8").tolist() == [5]
    assert np.frombuffer(raw[64:72], dtype="<f8").tolist() == [1.7]


def test_status_strings(lib):
    for code in range(8):
        s = aop.status_string(code)
        assert isinstance(s, str) and s and s != "unknown status"
    assert aop.status_string(99) == "unknown status"
    assert "sm_103a" in aop.version()


def test_no_device_is_an_error_not_a_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(aop.AopError) as ei:
        aop.Context(0)
    assert ei.value.code == 4   # AOP_ECUDA
    with pytest.raises(aop.AopError):
        aop.price_american(0, 100, 100, 0.05, 0.03, 0.2, 1.0, 64)


def test_workspace_bytes_is_host_arithmetic(lib):
    """aop_workspace_bytes needs no device: per-slot bytes times the count
    plus the launch's queue words; larger T needs more; stencils refused."""
    one = aop.workspace_bytes(aop.FFT_DF32, 1 << 13, 1)
    four = aop.workspace_bytes(aop.FFT_DF32, 1 << 13, 4)
    assert four - 8192 == 4 * (one - 8192) and one > 8192
    assert aop.workspace_bytes(aop.FFT_DF32, 1 << 17, 1) > one
    with pytest.raises(aop.AopError):
        aop.workspace_bytes(aop.STENCIL_FP64, 1 << 13, 1)
    with pytest.raises(aop.AopError):
        aop.workspace_bytes(aop.FFT_FP64, 0, 1)


def test_autotune_entry_points_check_arguments_on_the_host(lib):
    """Both tuner entry points refuse a null context, an empty sample and the
    plain stencil (which has no D&C schedule) before touching a device."""
    arr = aop.requests_array([dict(model=0, S0=100.0, K=100.0, r=0.05, q=0.03, sigma=0.2, expiry=1.0, T=64)])
    best = aop._Options()
    for args in ((None, 1, arr.ctypes.data, aop.FFT_DF32),
                 (None, 0, arr.ctypes.data, aop.FFT_DF32),
                 (None, 1, arr.ctypes.data, aop.STENCIL_FP64)):
        assert lib.aop_ctx_autotune(*args, ctypes.byref(best)) == 1                          # AOP_EINVAL
        assert lib.aop_ctx_autotune_flags(*args, aop.FLAG_NO_HELP, ctypes.byref(best)) == 1
