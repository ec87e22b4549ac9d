"""ctypes binding of the C ABI declared in ``include/ws.h``.

Argument marshalling only: every step of gridding and degridding runs in the
CUDA library.  There is no fallback -- if ``_build/libws_gb300.so`` is missing
or fails to load, :func:`load` raises.  PyTorch supplies device memory and
streams.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

WS_OK, WS_ERR_ARG, WS_ERR_UV_RANGE, WS_ERR_W_RANGE, WS_ERR_CUDA, WS_ERR_OOM, WS_ERR_TIMEOUT = range(7)
WS_FLAG_ASYNC = 1
WS_FLAG_NO_Z_OFFSET = 2
WS_FLAG_TIMING = 4
WS_FLAG_HERMITIAN = 8
WS_FLAG_DIVIDE_BY_N = 16
WS_FLAG_FP64 = 32
WS_FLAG_DETERMINISTIC = 64
STAGES = ("prep", "bin", "grid3d", "cols_inv", "rows_inv", "correct", "rows_fwd", "cols_fwd", "degrid3d")
STATUS_NAMES = {0: "WS_OK", 1: "WS_ERR_ARG", 2: "WS_ERR_UV_RANGE", 3: "WS_ERR_W_RANGE",
                4: "WS_ERR_CUDA", 5: "WS_ERR_OOM", 6: "WS_ERR_TIMEOUT"}

# every entry point declared in include/ws.h
EXPORTS = ("ws_plan", "ws_plan_original", "ws_degrid", "ws_grid", "ws_plan_bind_uvw", "ws_plan_tune",
           "ws_degrid_noalloc",
           "ws_plan_dropped", "ws_plan_info", "ws_plan_stats", "ws_destroy", "ws_batch_create", "ws_batch_grid", "ws_batch_degrid",
           "ws_batch_info", "ws_batch_branches", "ws_batch_destroy", "ws_last_error")


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("Np", ctypes.c_int32), ("W", ctypes.c_int32),
                ("Nw", ctypes.c_int32), ("t_lo", ctypes.c_int32), ("planes_per_chunk", ctypes.c_int32),
                ("x0", ctypes.c_double), ("n0", ctypes.c_double), ("nscale", ctypes.c_double),
                ("error_bound", ctypes.c_double), ("workspace_bytes", ctypes.c_int64),
                ("tile_rows", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("stage_ms", ctypes.c_double * len(STAGES)),
                ("stage_launches", ctypes.c_int64 * len(STAGES)),
                ("stage_bytes", ctypes.c_double * len(STAGES)),
                ("waits_timed_out", ctypes.c_int64)]

    def as_dict(self):
        return {"calls": self.calls, "kernel_launches": self.kernel_launches,
                "stage_ms": {n: self.stage_ms[i] for i, n in enumerate(STAGES)},
                "stage_launches": {n: self.stage_launches[i] for i, n in enumerate(STAGES)},
                "stage_bytes": {n: self.stage_bytes[i] for i, n in enumerate(STAGES)},
                "waits_timed_out": self.waits_timed_out}


class Instance(ctypes.Structure):
    """ws_instance_t: one problem of a batch."""
    _fields_ = [("N", ctypes.c_int32), ("fov", ctypes.c_double), ("w_min", ctypes.c_double),
                ("w_max", ctypes.c_double), ("M", ctypes.c_int64)]


class WsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB) -> ctypes.CDLL:
    """Load the library once; raise if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
    lib.ws_plan.argtypes = [ctypes.POINTER(vp), i32, dbl, i32, dbl, dbl, dbl, u32]
    lib.ws_plan_original.argtypes = [ctypes.POINTER(vp), i32, dbl, i32, dbl, dbl, dbl, i32, u32]
    lib.ws_degrid.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.ws_grid.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.ws_plan_bind_uvw.argtypes = [vp, vp, i64, vp]
    lib.ws_plan_tune.argtypes = [vp, vp, vp, vp, i64, ctypes.c_char_p, vp, ctypes.POINTER(i32)]
    lib.ws_degrid_noalloc.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.ws_plan_dropped.argtypes = [vp, ctypes.POINTER(i64)]
    lib.ws_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.ws_plan_stats.argtypes = [vp, ctypes.POINTER(Stats), i32]
    lib.ws_destroy.argtypes = [vp]
    pp = ctypes.POINTER(vp)
    lib.ws_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Instance), dbl, i32, i32, i64, u32]
    lib.ws_batch_grid.argtypes = [vp, pp, pp, pp, vp]
    lib.ws_batch_degrid.argtypes = [vp, pp, pp, pp, vp]
    lib.ws_batch_info.argtypes = [vp, i32, ctypes.POINTER(PlanInfo), ctypes.POINTER(i32)]
    lib.ws_batch_branches.argtypes = [vp, ctypes.POINTER(i32)]
    lib.ws_batch_destroy.argtypes = [vp]
    lib.ws_last_error.argtypes = []
    lib.ws_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "ws_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != WS_OK:
        raise WsError(status, load().ws_last_error().decode(errors="replace"))


# -- the C entry points under their own names --------------------------------

def ws_plan(N: int, x0: float, W: int, fov: float, w_min: float, w_max: float, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().ws_plan(ctypes.byref(h), N, x0, W, fov, w_min, w_max, flags))
    return h.value


def ws_plan_original(N: int, x0: float, W: int, fov: float, w_min: float, w_max: float, Nw: int,
                     flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().ws_plan_original(ctypes.byref(h), N, x0, W, fov, w_min, w_max, Nw, flags))
    return h.value


def ws_degrid(plan: int, image_ptr: int, uvw_ptr: int, M: int, vis_ptr: int, stream: int = 0) -> int:
    """Returns the status (WS_ERR_W_RANGE / WS_ERR_UV_RANGE are not raised)."""
    st = load().ws_degrid(plan, image_ptr, uvw_ptr, M, vis_ptr, stream)
    if st not in (WS_OK, WS_ERR_UV_RANGE, WS_ERR_W_RANGE):
        _check(st)
    return st


def ws_grid(plan: int, uvw_ptr: int, vis_ptr: int, M: int, dirty_ptr: int, stream: int = 0) -> int:
    st = load().ws_grid(plan, uvw_ptr, vis_ptr, M, dirty_ptr, stream)
    if st not in (WS_OK, WS_ERR_UV_RANGE, WS_ERR_W_RANGE):
        _check(st)
    return st


def ws_plan_bind_uvw(plan: int, uvw_ptr: int, M: int, stream: int = 0) -> None:
    """Pre-process and bin a uvw set once for later calls with the same pointer and M (0 unbinds)."""
    _check(load().ws_plan_bind_uvw(plan, uvw_ptr, M, stream))


def ws_plan_tune(plan: int, uvw_ptr: int, vis_ptr: int, image_ptr: int, M: int, cache_path: str | None = None,
                 stream: int = 0) -> int:
    """Time the gridding tile's row counts on this data, keep the fastest; returns it."""
    rows = ctypes.c_int32()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(load().ws_plan_tune(plan, uvw_ptr, vis_ptr, image_ptr, M, path, stream, ctypes.byref(rows)))
    return rows.value


def ws_degrid_noalloc(plan: int, image_ptr: int, uvw_ptr: int, M: int, vis_ptr: int, stream: int = 0) -> int:
    """Degridding with no device allocation (scratch in a fixed 64 MiB device array)."""
    st = load().ws_degrid_noalloc(plan, image_ptr, uvw_ptr, M, vis_ptr, stream)
    if st not in (WS_OK, WS_ERR_UV_RANGE, WS_ERR_W_RANGE):
        _check(st)
    return st


def ws_plan_dropped(plan: int) -> int:
    n = ctypes.c_int64()
    _check(load().ws_plan_dropped(plan, ctypes.byref(n)))
    return n.value


def ws_plan_info(plan: int) -> PlanInfo:
    info = PlanInfo()
    _check(load().ws_plan_info(plan, ctypes.byref(info)))
    return info


def ws_plan_stats(plan: int, reset: bool = False) -> Stats:
    st = Stats()
    _check(load().ws_plan_stats(plan, ctypes.byref(st), 1 if reset else 0))
    return st


def ws_destroy(plan: int) -> None:
    _check(load().ws_destroy(plan))


def _ptrs(values):
    arr = (ctypes.c_void_p * len(values))(*[int(v) for v in values])
    return arr


def ws_batch_create(instances, x0: float, W: int, branches: int = 0, workspace_bytes: int = 0,
                    flags: int = 0) -> int:
    """instances: sequence of (N, fov, w_min, w_max, M)."""
    arr = (Instance * len(instances))(*[Instance(int(N), float(fov), float(a), float(b), int(M))
                                        for (N, fov, a, b, M) in instances])
    h = ctypes.c_void_p()
    _check(load().ws_batch_create(ctypes.byref(h), len(instances), arr, x0, W, branches, workspace_bytes, flags))
    return h.value


def ws_batch_grid(batch: int, uvw_ptrs, vis_ptrs, dirty_ptrs, stream: int = 0) -> int:
    st = load().ws_batch_grid(batch, _ptrs(uvw_ptrs), _ptrs(vis_ptrs), _ptrs(dirty_ptrs), stream)
    if st not in (WS_OK, WS_ERR_UV_RANGE, WS_ERR_W_RANGE):
        _check(st)
    return st


def ws_batch_degrid(batch: int, image_ptrs, uvw_ptrs, vis_ptrs, stream: int = 0) -> int:
    st = load().ws_batch_degrid(batch, _ptrs(image_ptrs), _ptrs(uvw_ptrs), _ptrs(vis_ptrs), stream)
    if st not in (WS_OK, WS_ERR_UV_RANGE, WS_ERR_W_RANGE):
        _check(st)
    return st


def ws_batch_info(batch: int, i: int):
    info, branch = PlanInfo(), ctypes.c_int32()
    _check(load().ws_batch_info(batch, i, ctypes.byref(info), ctypes.byref(branch)))
    return info, branch.value


def ws_batch_branches(batch: int) -> int:
    k = ctypes.c_int32()
    _check(load().ws_batch_branches(batch, ctypes.byref(k)))
    return k.value


def ws_batch_destroy(batch: int) -> None:
    _check(load().ws_batch_destroy(batch))


def ws_last_error() -> str:
    return load().ws_last_error().decode(errors="replace")
