"""Batches of independent problems (``ws_batch_*`` in ``include/ws.h``).

Each instance has its own image size, field, w-range and visibility count;
x0 and W are shared.  Only marshalling happens here: lists of device tensors
become host arrays of device pointers, and the CUDA library runs every
instance (on parallel branches, captured once into a CUDA graph and replayed
by later calls with the same tensors).
"""
from __future__ import annotations

import torch

from . import _lib


class Batch:
    """``instances``: sequence of (N, fov, w_min, w_max, M)."""

    def __init__(self, instances, x0: float, W: int, branches: int = 0, workspace_bytes: int = 0,
                 flags: int = 0, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.instances = [tuple(i) for i in instances]
        with torch.cuda.device(self.device):
            self.handle = _lib.ws_batch_create(self.instances, float(x0), int(W), int(branches),
                                               int(workspace_bytes), int(flags))
        self.info = [_lib.ws_batch_info(self.handle, i)[0] for i in range(len(self.instances))]
        self.last_status = _lib.WS_OK

    def __len__(self):
        return len(self.instances)

    @property
    def branches(self) -> int:
        return _lib.ws_batch_branches(self.handle)

    def branch_of(self, i: int) -> int:
        return _lib.ws_batch_info(self.handle, i)[1]

    def _check(self, tensors, dtype, shapes, name):
        if len(tensors) != len(self.instances):
            raise ValueError(f"{name}: need {len(self.instances)} tensors, got {len(tensors)}")
        for i, (t, shape) in enumerate(zip(tensors, shapes)):
            if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() \
                    or t.device != self.device:
                raise ValueError(f"{name}[{i}]: need contiguous {dtype} {tuple(shape)} on {self.device}, "
                                 f"got {t.dtype} {tuple(t.shape)} on {t.device}")

    def _stream(self, stream):
        return (torch.cuda.current_stream(self.device) if stream is None else stream).cuda_stream

    def grid(self, uvw, vis, out=None, stream=None):
        """Algorithm 5 on every instance: lists of uvw (M_i, 3) float64 and vis (M_i,) complex64."""
        Ms = [inst[4] for inst in self.instances]
        Ns = [inst[0] for inst in self.instances]
        self._check(uvw, torch.float64, [(M, 3) for M in Ms], "uvw")
        self._check(vis, torch.complex64, [(M,) for M in Ms], "vis")
        if out is None:
            out = [torch.empty(N, N, dtype=torch.complex64, device=self.device) for N in Ns]
        self._check(out, torch.complex64, [(N, N) for N in Ns], "out")
        self.last_status = _lib.ws_batch_grid(self.handle, [t.data_ptr() for t in uvw],
                                              [t.data_ptr() for t in vis], [t.data_ptr() for t in out],
                                              self._stream(stream))
        return out

    def degrid(self, images, uvw, out=None, stream=None):
        """Algorithm 6 on every instance: lists of images (N_i, N_i) complex64 and uvw."""
        Ms = [inst[4] for inst in self.instances]
        Ns = [inst[0] for inst in self.instances]
        self._check(images, torch.complex64, [(N, N) for N in Ns], "images")
        self._check(uvw, torch.float64, [(M, 3) for M in Ms], "uvw")
        if out is None:
            out = [torch.empty(M, dtype=torch.complex64, device=self.device) for M in Ms]
        self._check(out, torch.complex64, [(M,) for M in Ms], "out")
        self.last_status = _lib.ws_batch_degrid(self.handle, [t.data_ptr() for t in images],
                                                [t.data_ptr() for t in uvw], [t.data_ptr() for t in out],
                                                self._stream(stream))
        return out

    def close(self):
        if getattr(self, "handle", None):
            _lib.ws_batch_destroy(self.handle)
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
