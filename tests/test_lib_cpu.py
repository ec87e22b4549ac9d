"""The C-ABI library builds, loads and exports what include/ws.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2101_11172_gb300 import _lib
from paper_2101_11172_gb300.build import LIB, ROOT, build


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ws.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ws_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ws_plan", "ws_degrid", "ws_grid", "ws_destroy"):
        assert required in names
    assert set(names) == set(_lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {LIB}").read()
    exported = set(re.findall(r" T (ws_\w+)", out))
    assert set(declared_functions()) <= exported


def test_sm103a_only_build_flags():
    from paper_2101_11172_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_argument_validation_needs_no_device(lib):
    # Parameter checks happen before any CUDA call.
    h = ctypes.c_void_p()
    bad = [(15, 0.25, 7, 0.2, -1, 1), (64, 0.6, 7, 0.2, -1, 1), (64, 0.25, 0, 0.2, -1, 1),
           (64, 0.25, 13, 0.2, -1, 1), (64, 0.25, 7, 1.5, -1, 1), (64, 0.25, 7, 0.2, 2, 1),
           (64, 0.25, 7, 0.2, float("nan"), 1), (64, 0.25, 7, 0.2, -1e7, 1e7)]
    for args in bad:
        st = lib.ws_plan(ctypes.byref(h), *args, 0)
        assert st == _lib.WS_ERR_ARG, args
        assert h.value is None
        assert _lib.ws_last_error()
    assert lib.ws_plan(None, 64, 0.25, 7, 0.2, -1, 1, 0) == _lib.WS_ERR_ARG
    assert lib.ws_plan(ctypes.byref(h), 64, 0.25, 7, 0.2, -1, 1, 1 << 8) == _lib.WS_ERR_ARG
    assert lib.ws_grid(None, None, None, 0, None, None) == _lib.WS_ERR_ARG
    assert lib.ws_degrid(None, None, None, 0, None, None) == _lib.WS_ERR_ARG
    assert lib.ws_plan_info(None, None) == _lib.WS_ERR_ARG
    assert lib.ws_plan_bind_uvw(None, None, 0, None) == _lib.WS_ERR_ARG
    # FP64 plans: W up to 14, power-of-two N' only, not for the original method
    assert lib.ws_plan(ctypes.byref(h), 64, 0.25, 15, 0.2, -1, 1, _lib.WS_FLAG_FP64) == _lib.WS_ERR_ARG
    assert lib.ws_plan(ctypes.byref(h), 200, 0.25, 7, 0.2, -1, 1, _lib.WS_FLAG_FP64) == _lib.WS_ERR_ARG
    assert "power-of-two" in _lib.ws_last_error()
    assert lib.ws_plan(ctypes.byref(h), 64, 0.25, 13, 0.2, -1, 1, 0) == _lib.WS_ERR_ARG
    assert lib.ws_plan_original(ctypes.byref(h), 64, 0.25, 7, 0.2, -1, 1, 20, _lib.WS_FLAG_FP64) == _lib.WS_ERR_ARG
    assert lib.ws_destroy(None) == _lib.WS_OK


def test_missing_library_fails_loudly(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_batch_argument_validation_needs_no_device(lib):
    h = ctypes.c_void_p()
    one = (_lib.Instance * 1)(_lib.Instance(64, 0.2, -1.0, 1.0, 100))
    # no instances, too many branches, negative workspace, flags a batch does not take
    assert lib.ws_batch_create(ctypes.byref(h), 0, one, 0.25, 7, 0, 0, 0) == _lib.WS_ERR_ARG
    assert lib.ws_batch_create(ctypes.byref(h), 1, one, 0.25, 7, 9, 0, 0) == _lib.WS_ERR_ARG
    assert lib.ws_batch_create(ctypes.byref(h), 1, one, 0.25, 7, 0, -1, 0) == _lib.WS_ERR_ARG
    assert lib.ws_batch_create(ctypes.byref(h), 1, one, 0.25, 7, 0, 0, _lib.WS_FLAG_TIMING) == _lib.WS_ERR_ARG
    assert lib.ws_batch_create(None, 1, one, 0.25, 7, 0, 0, 0) == _lib.WS_ERR_ARG
    neg = (_lib.Instance * 1)(_lib.Instance(64, 0.2, -1.0, 1.0, -5))
    assert lib.ws_batch_create(ctypes.byref(h), 1, neg, 0.25, 7, 0, 0, 0) == _lib.WS_ERR_ARG
    assert "instance 0" in _lib.ws_last_error()
    assert h.value is None
    assert lib.ws_batch_grid(None, None, None, None, None) == _lib.WS_ERR_ARG
    assert lib.ws_batch_degrid(None, None, None, None, None) == _lib.WS_ERR_ARG
    assert lib.ws_batch_info(None, 0, None, None) == _lib.WS_ERR_ARG
    assert lib.ws_batch_destroy(None) == _lib.WS_OK
