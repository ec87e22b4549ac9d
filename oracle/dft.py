"""Exact operator by brute force (Eq. fourier_visibility and its adjoint), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

``dft_degrid`` and ``dft_grid`` call the plain-C loops of ``oracle/dft.c``
(compiled on first use with gcc and OpenMP into ``oracle/_build/``);
``dft_*_numpy`` restate the same sums with numpy for micro inputs, so the C
code can be checked against a second transcription of the definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .geometry import Geometry, n_minus_one

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dft.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_dft.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/dft.c (portable flags only) and return the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.oracle_dft_degrid.argtypes = [i64, d, i64, d, d, d]
        lib.oracle_dft_grid.argtypes = [i64, d, d, i64, d, d]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pixel_lmn(geom: Geometry, rows=None, cols=None):
    """(l, m, n-1) for image pixels [i, j]; all pixels if rows/cols are None."""
    lm = geom.pixel_lm()
    if rows is None:
        ii, jj = np.meshgrid(np.arange(geom.N), np.arange(geom.N), indexing="ij")
        rows, cols = ii.ravel(), jj.ravel()
    l = lm[np.asarray(cols)]
    m = lm[np.asarray(rows)]
    return np.ascontiguousarray(np.stack([l, m, n_minus_one(l, m)], 1))


def dft_degrid(uvw, lmn, f):
    """V_k = sum_p f_p exp(-2 pi i (u l + v m + w (n-1)))."""
    lib = _load()
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    lmn = np.ascontiguousarray(lmn, dtype=np.float64)
    f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128).ravel())
    out = np.zeros(uvw.shape[0], dtype=np.complex128)
    lib.oracle_dft_degrid(uvw.shape[0], _ptr(uvw), lmn.shape[0], _ptr(lmn),
                          _ptr(f.view(np.float64)), _ptr(out.view(np.float64)))
    return out


def dft_grid(uvw, vis, lmn):
    """d_p = sum_k V_k exp(+2 pi i (u l + v m + w (n-1)))."""
    lib = _load()
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    lmn = np.ascontiguousarray(lmn, dtype=np.float64)
    vis = np.ascontiguousarray(np.asarray(vis, dtype=np.complex128))
    out = np.zeros(lmn.shape[0], dtype=np.complex128)
    lib.oracle_dft_grid(uvw.shape[0], _ptr(uvw), _ptr(vis.view(np.float64)), lmn.shape[0],
                        _ptr(lmn), _ptr(out.view(np.float64)))
    return out


def _phase_matrix(uvw, lmn):
    uvw = np.asarray(uvw, dtype=np.float64)
    lmn = np.asarray(lmn, dtype=np.float64)
    return uvw @ lmn.T                                       # (M, P) turns


def dft_degrid_numpy(uvw, lmn, f):
    return np.exp(-2j * np.pi * _phase_matrix(uvw, lmn)) @ np.asarray(f, np.complex128).ravel()


def dft_grid_numpy(uvw, vis, lmn):
    return np.exp(2j * np.pi * _phase_matrix(uvw, lmn)).T @ np.asarray(vis, np.complex128)
