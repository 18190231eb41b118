"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-only queries and error paths behave."""
import ctypes
import os
import re

import pytest

import paper_2601_12209_gb300 as gb
from paper_2601_12209_gb300 import _build, abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return abi.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gbfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbfft_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared_functions() == sorted(abi.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_host_queries(lib):
    assert "sm_103a" in abi.gbfft_version()
    assert abi.gbfft_radix_plan(512) == [8, 8, 8]
    assert abi.gbfft_radix_plan(1024) == [16, 8, 8]
    assert abi.gbfft_radix_plan(60) == [4, 3, 5]
    assert abi.gbfft_radix_plan(256) == [16, 16]
    for n in (2, 3, 5, 8, 16, 32, 48, 60, 64, 80, 96, 120, 128, 160, 192, 256, 512, 1024):
        assert abi.gbfft_supported_length(n), n
        prod = 1
        for r in abi.gbfft_radix_plan(n):
            assert r in (2, 3, 4, 5, 8, 16)
            prod *= r
        assert prod == n
    for n in (1, 7, 11, 14, 2048, 1000):
        assert not abi.gbfft_supported_length(n), n
    with pytest.raises(abi.GbfftError):
        abi.gbfft_radix_plan(7)
    for code in range(-10, 1):
        assert abi.strerror(code) and abi.strerror(code) != "unknown error"


def test_invalid_arguments_rejected_before_device(lib):
    h = ctypes.c_void_p()
    f = lib.gbfft_plan_create
    assert f(None, 8, 8, 8, 0, 0, 1, 0) == abi.GBFFT_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 1, 8, 8, 0, 0, 1, 0) == abi.GBFFT_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 7, 0, 1, 0) == abi.GBFFT_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 0, 5, 1, 0) == abi.GBFFT_ERR_INVALID_ARG  # no such dtype
    for dt in (abi.GBFFT_FP16_SPLIT, abi.GBFFT_BF16_SPLIT, abi.GBFFT_FP16_SPLIT_TC5, abi.GBFFT_BF16_SPLIT_TC5):
        assert f(ctypes.byref(h), 9, 8, 8, abi.GBFFT_R2C, dt, 1, 0) == abi.GBFFT_ERR_INVALID_ARG  # odd nx
    assert f(ctypes.byref(h), 8, 8, 8, 0, 0, 0, 0) == abi.GBFFT_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 0, 0, 1, 1 << 20) == abi.GBFFT_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 0, 0, 1, abi.GBFFT_SLAB | abi.GBFFT_TRANSPOSED_OUT) == abi.GBFFT_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 9, 8, 8, 1, 0, 1, 0) == abi.GBFFT_ERR_INVALID_ARG  # odd nx for R2C
    assert f(ctypes.byref(h), 7, 8, 8, 0, 0, 1, 0) == abi.GBFFT_ERR_UNSUPPORTED_SIZE
    assert f(ctypes.byref(h), 8, 8, 2048, 0, 0, 1, 0) == abi.GBFFT_ERR_UNSUPPORTED_SIZE
    assert h.value is None
    dims = (ctypes.c_int * 3)(32, 32, 32)
    mk = lib.gbfft_many_create
    assert mk(ctypes.byref(h), 1, dims, abi.GBFFT_R2C, abi.GBFFT_FP32, 0) == abi.GBFFT_ERR_INVALID_ARG  # C2C only
    assert mk(ctypes.byref(h), 1, dims, abi.GBFFT_C2C, abi.GBFFT_FP16_SPLIT, 0) == abi.GBFFT_ERR_INVALID_ARG
    assert mk(ctypes.byref(h), 0, dims, abi.GBFFT_C2C, abi.GBFFT_FP32, 0) == abi.GBFFT_ERR_INVALID_ARG
    assert h.value is None
    assert lib.gbfft_many_autotune(None, None) == abi.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_exec(None, 0, None, None, None) == abi.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_workspace_size(None, None) == abi.GBFFT_ERR_INVALID_ARG
    lib.gbfft_plan_destroy(None)


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.gbfft_plan_create(ctypes.byref(h), 8, 8, 8, 0, 0, 1, 0) == abi.GBFFT_ERR_NO_DEVICE
    with pytest.raises(abi.GbfftError):
        gb.Plan(8, 8, 8)
