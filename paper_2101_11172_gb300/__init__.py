"""GB300-native improved W-stacking gridder/degridder (Ye, Gull, Tan & Nikolic 2021).

The computation lives in the CUDA library ``_build/libws_gb300.so`` behind the
C ABI of ``include/ws.h``; :mod:`._lib` binds it with ctypes and
:mod:`.wstack` wraps it for PyTorch device tensors.
"""
from ._lib import (WS_FLAG_ASYNC, WS_FLAG_DETERMINISTIC, WS_FLAG_DIVIDE_BY_N, WS_FLAG_FP64, WS_FLAG_HERMITIAN,  # noqa: F401
                   WS_FLAG_NO_Z_OFFSET, WS_FLAG_TIMING, WsError, load)

__all__ = ["Plan", "WsError", "load", "WS_FLAG_ASYNC", "WS_FLAG_DETERMINISTIC", "WS_FLAG_DIVIDE_BY_N", "WS_FLAG_FP64",
           "WS_FLAG_HERMITIAN",
           "WS_FLAG_NO_Z_OFFSET", "WS_FLAG_TIMING"]


def __getattr__(name):
    if name == "Plan":
        from .wstack import Plan
        return Plan
    raise AttributeError(name)
