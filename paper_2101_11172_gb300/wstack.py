"""PyTorch-facing wrapper of the C ABI: device tensors in, device tensors out.

Only marshalling happens here (shapes, dtypes, pointers, the current CUDA
stream); the computation is the CUDA library's.  Tensors must already live on
the plan's device: complex64 images (N, N) with rows along m and columns along
l, complex64 visibilities (M,), float64 uvw (M, 3) in wavelengths; complex128
images and visibilities for plans made with WS_FLAG_FP64.
"""
from __future__ import annotations

import torch

from . import _lib


class Plan:
    """Improved W-stacking plan (``ws_plan``); see ``include/ws.h``."""

    def __init__(self, N: int, x0: float, W: int, fov: float, w_min: float, w_max: float,
                 flags: int = 0, device=None, original_bins: int = 0):
        """``original_bins > 0`` builds the original W-stacking plan (``ws_plan_original``)."""
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            if original_bins > 0:
                self.handle = _lib.ws_plan_original(int(N), float(x0), int(W), float(fov), float(w_min),
                                                    float(w_max), int(original_bins), int(flags))
            else:
                self.handle = _lib.ws_plan(int(N), float(x0), int(W), float(fov), float(w_min),
                                           float(w_max), int(flags))
        info = _lib.ws_plan_info(self.handle)
        self.N, self.Np, self.W, self.Nw = info.N, info.Np, info.W, info.Nw
        self.t_lo, self.planes_per_chunk = info.t_lo, info.planes_per_chunk
        self.x0, self.n0, self.nscale = info.x0, info.n0, info.nscale
        self.error_bound = info.error_bound
        self.flags = flags
        self.cdtype = torch.complex128 if flags & _lib.WS_FLAG_FP64 else torch.complex64
        self.last_status = _lib.WS_OK
        self._bound = None             # (uvw tensor, its version when bound)

    @property
    def tile_rows(self) -> int:
        return _lib.ws_plan_info(self.handle).tile_rows

    def tune(self, uvw: torch.Tensor, vis: torch.Tensor, image: torch.Tensor, cache_path: str | None = None,
             stream=None) -> int:
        """``ws_plan_tune``: time the gridding tile's row counts on this data and keep the fastest."""
        M = uvw.shape[0]
        self._check(uvw, torch.float64, (M, 3), "uvw")
        self._check(vis, torch.complex64, (M,), "vis")
        self._check(image, torch.complex64, (self.N, self.N), "image")
        rows = _lib.ws_plan_tune(self.handle, uvw.data_ptr(), vis.data_ptr(), image.data_ptr(), M, cache_path,
                                 self._stream(stream))
        self._bound = None
        return rows

    @property
    def workspace_bytes(self) -> int:
        return _lib.ws_plan_info(self.handle).workspace_bytes

    def _stream(self, stream):
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        return s.cuda_stream

    def _check(self, t: torch.Tensor, dtype, shape, name):
        if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() \
                or t.device != self.device:
            raise ValueError(f"{name}: need contiguous {dtype} {tuple(shape)} on {self.device}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")

    def bind(self, uvw: torch.Tensor | None, stream=None) -> None:
        """Pre-process and bin ``uvw`` once (``ws_plan_bind_uvw``): later calls with this
        tensor skip that work.  The plan keeps a reference to the tensor, so its memory
        stays allocated; an in-place change to it is noticed (through the tensor's
        version counter) and the set is bound again on the next call.  ``None`` unbinds."""
        if uvw is None:
            _lib.ws_plan_bind_uvw(self.handle, 0, 0, self._stream(stream))
            self._bound = None
            return
        self._check(uvw, torch.float64, (uvw.shape[0], 3), "uvw")
        _lib.ws_plan_bind_uvw(self.handle, uvw.data_ptr(), uvw.shape[0], self._stream(stream))
        self._bound = (uvw, uvw._version)

    def _refresh_binding(self, uvw: torch.Tensor, stream) -> None:
        b = self._bound
        if b is not None and b[0].data_ptr() == uvw.data_ptr() and b[0].shape == uvw.shape \
                and b[0]._version != b[1]:
            self.bind(b[0], stream)

    def degrid(self, image: torch.Tensor, uvw: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
        """Algorithm 6: model image -> visibilities (``ws_degrid``)."""
        M = uvw.shape[0]
        self._refresh_binding(uvw, stream)
        self._check(image, self.cdtype, (self.N, self.N), "image")
        self._check(uvw, torch.float64, (M, 3), "uvw")
        if out is None:
            out = torch.empty(M, dtype=self.cdtype, device=self.device)
        self._check(out, self.cdtype, (M,), "out")
        self.last_status = _lib.ws_degrid(self.handle, image.data_ptr(), uvw.data_ptr(), M,
                                          out.data_ptr(), self._stream(stream))
        return out

    def grid(self, uvw: torch.Tensor, vis: torch.Tensor, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
        """Algorithm 5: visibilities -> dirty image (``ws_grid``)."""
        M = uvw.shape[0]
        self._refresh_binding(uvw, stream)
        self._check(uvw, torch.float64, (M, 3), "uvw")
        self._check(vis, self.cdtype, (M,), "vis")
        if out is None:
            out = torch.empty(self.N, self.N, dtype=self.cdtype, device=self.device)
        self._check(out, self.cdtype, (self.N, self.N), "out")
        self.last_status = _lib.ws_grid(self.handle, uvw.data_ptr(), vis.data_ptr(), M,
                                        out.data_ptr(), self._stream(stream))
        return out

    def stats(self, reset: bool = False) -> dict:
        """Call counters and (WS_FLAG_TIMING plans) per-stage device milliseconds."""
        return _lib.ws_plan_stats(self.handle, reset).as_dict()

    def dropped(self) -> int:
        return _lib.ws_plan_dropped(self.handle)

    def close(self):
        self._bound = None
        if getattr(self, "handle", None):
            _lib.ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
