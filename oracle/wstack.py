"""Least-misfit gridding/degridding and improved W-stacking, step by step, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Normalisation (a reading; the paper's 1/M natural weighting and the
``2 l_max`` / ``4 l_max m_max`` factors of Section 3.1 and Section 5.2 are
scalars a caller applies): every operator here is a plain sum, so that

* degridding approximates ``V_k = sum_{i,j} f[i,j] exp(-2 pi i (u_k l_j + v_k m_i + w_k (n_ij - 1)))``,
* gridding approximates ``d[i,j] = sum_k V_k exp(+2 pi i (u_k l_j + v_k m_i + w_k (n_ij - 1)))``,

and the two are exact adjoints under the plain complex inner products
(Eq. equal_norms and the adjoint pair of Algorithms 5 and 6).

Grid indices are kept modulo N' ("wrapped"): a grid point r is stored at
``r mod N'``.  Because ``exp(2 pi i r j / N')`` is N'-periodic in r, the sum
over all integers r in Eq. gridded-dirty-map equals the N'-point inverse DFT
of the wrapped grid, so no visibility ever falls off the grid and the centred
transforms need no sign factors.
"""
from __future__ import annotations

import numpy as np

from .geometry import Geometry, first_tap
from .lmfit import LeastMisfit, interpolated_h


# -- one dimension: Algorithms 1 and 2 --------------------------------------

def grid_1d(lm: LeastMisfit, Np: int, N: int, up, V):
    """Algorithm 1: d(x_j), j = -N/2..N/2-1, from visibilities V at u'."""
    W = lm.W
    r0, nu = first_tap(up, W)
    c = lm.weights(nu)                                          # (M, W)
    G = np.zeros(Np, dtype=np.complex128)
    for i in range(W):                                          # step (1): spread
        np.add.at(G, (r0 + i) % Np, V * c[:, i])
    img = np.fft.ifft(G) * Np                                   # step (2): inverse FFT
    j = np.arange(N) - N // 2
    return lm.h(j / Np) * img[j % Np]                           # steps (3), (4): crop, x h


def degrid_1d(lm: LeastMisfit, Np: int, f, up):
    """Algorithm 2: visibilities at u' from an N-pixel model f (exact adjoint of grid_1d)."""
    N = f.shape[0]
    W = lm.W
    j = np.arange(N) - N // 2
    padded = np.zeros(Np, dtype=np.complex128)                  # step (1): zero pad
    padded[j % Np] = lm.h(j / Np) * f                           # step (2): x h
    F = np.fft.fft(padded)                                      # step (3): FFT
    r0, nu = first_tap(up, W)
    c = lm.weights(nu)
    out = np.zeros(np.shape(up), dtype=np.complex128)
    for i in range(W):                                          # step (4): correlate with C
        out += F[(r0 + i) % Np] * c[:, i]
    return out


# -- three dimensions: Algorithms 5 and 6 ------------------------------------

def _taps(geom: Geometry, lm: LeastMisfit, uvw):
    up, vp, wp = geom.scaled(uvw)
    r0, nux = first_tap(up, geom.W)
    s0, nuy = first_tap(vp, geom.W)
    t0, nuz = first_tap(wp, geom.W)
    return (r0, s0, t0), (lm.weights(nux), lm.weights(nuy), lm.weights(nuz))


def prephase(geom: Geometry, w):
    """exp(2 pi i w (n0 - 1)) of Eq. gridded_vis; its conjugate closes Algorithm 6."""
    turns = np.asarray(w, dtype=np.float64) * (geom.n0 - 1.0)
    turns = turns - np.rint(turns)
    return np.exp(2j * np.pi * turns)


_CORRECTIONS = {}


def correction(geom: Geometry, lm: LeastMisfit, with_hz: bool = True):
    """h_x(x) h_y(y) h_z(z(x, y)) on the N x N image (Algorithm 5 step 5).

    Section 5.3: the product is computed once for all image points, with
    h_z(z) taken by high-degree interpolation in a uniform table of h.  It
    depends on the image geometry only (not on the w-range), so it is kept
    per geometry.
    """
    key = (geom.N, geom.Np, geom.x0, geom.fov, geom.nscale, geom.n0, lm.W, lm.x0, lm.beta.tobytes(), with_hz)
    if key not in _CORRECTIONS:
        hx = lm.h(geom.pixel_x())
        out = hx[None, :] * hx[:, None]
        if with_hz:
            out = out * interpolated_h(lm)(geom.pixel_z())
        if len(_CORRECTIONS) > 8:
            _CORRECTIONS.clear()
        _CORRECTIONS[key] = out
    return _CORRECTIONS[key]


def _crop_index(geom: Geometry):
    return (np.arange(geom.N) - geom.N // 2) % geom.Np


def _check_w(geom: Geometry, t0):
    if t0.size and (t0.min() < geom.t_lo or t0.max() + geom.W - 1 > geom.t_hi):
        raise ValueError("w outside the plan's w-range")


def grid(geom: Geometry, lm: LeastMisfit, uvw, vis, with_hz: bool = True):
    """Algorithm 5: dirty image d[i, j] (i along m, j along l) from visibilities."""
    W, Np = geom.W, geom.Np
    (r0, s0, t0), (cx, cy, cz) = _taps(geom, lm, uvw)
    _check_w(geom, t0)
    Vt = np.asarray(vis, dtype=np.complex128) * prephase(geom, np.asarray(uvw)[:, 2])  # step 2
    z = geom.pixel_z()
    idx = _crop_index(geom)
    acc = np.zeros((geom.N, geom.N), dtype=np.complex128)
    for t in range(geom.t_lo, geom.t_hi + 1):
        sel = np.nonzero((t >= t0) & (t < t0 + W))[0]
        G = np.zeros((Np, Np), dtype=np.complex128)
        if sel.size:
            wz = cz[sel, t - t0[sel]] * Vt[sel]                 # step 2: C_z(t - w')
            for b in range(W):                                  # step 3a: C_x C_y onto (s, r)
                rows = (s0[sel] + b) % Np
                wb = wz * cy[sel, b]
                for a in range(W):
                    np.add.at(G, (rows, (r0[sel] + a) % Np), wb * cx[sel, a])
        P = np.fft.ifft2(G) * (Np * Np)                         # step 3b: inverse 2-D FFT
        crop = P[np.ix_(idx, idx)]                              # step 3c: crop
        tz = t * z
        acc += crop * np.exp(2j * np.pi * (tz - np.rint(tz)))   # steps 3d, 4
    return correction(geom, lm, with_hz) * acc                  # step 5


def degrid(geom: Geometry, lm: LeastMisfit, image, uvw, with_hz: bool = True):
    """Algorithm 6: visibilities from an N x N model image (transpose of grid)."""
    W, Np = geom.W, geom.Np
    (r0, s0, t0), (cx, cy, cz) = _taps(geom, lm, uvw)
    _check_w(geom, t0)
    corrected = correction(geom, lm, with_hz) * np.asarray(image, dtype=np.complex128)  # step 2
    z = geom.pixel_z()
    idx = _crop_index(geom)
    out = np.zeros(r0.shape, dtype=np.complex128)
    for t in range(geom.t_lo, geom.t_hi + 1):
        sel = np.nonzero((t >= t0) & (t < t0 + W))[0]
        if not sel.size:
            continue
        tz = t * z
        Q = np.zeros((Np, Np), dtype=np.complex128)
        Q[np.ix_(idx, idx)] = corrected * np.exp(-2j * np.pi * (tz - np.rint(tz)))  # 3a, 3b
        F = np.fft.fft2(Q)                                      # step 3c
        acc = np.zeros(sel.size, dtype=np.complex128)
        for b in range(W):                                      # step 4: 3-D correlation
            rows = (s0[sel] + b) % Np
            for a in range(W):
                acc += F[rows, (r0[sel] + a) % Np] * (cx[sel, a] * cy[sel, b])
        out[sel] += acc * cz[sel, t - t0[sel]]
    return out * np.conj(prephase(geom, np.asarray(uvw)[:, 2]))  # step 5


# -- the original W-stacking: Algorithms 3 and 4 -----------------------------

def _bins(geom: Geometry, uvw):
    """Nearest bin t = floor(w' + 1/2) of each visibility (Algorithm 3 step 2)."""
    t = np.floor(np.asarray(uvw, dtype=np.float64)[:, 2] * geom.nscale + 0.5).astype(np.int64)
    if t.size and (t.min() < geom.t_lo or t.max() > geom.t_hi):
        raise ValueError("w outside the plan's w-range")
    return t


def grid_original(geom: Geometry, lm: LeastMisfit, uvw, vis):
    """Algorithm 3: per w-bin 2-D gridding, inverse FFT, crop and exp(2 pi i w[t] (n - 1));
    the sum over bins times the 2-D gridding correction h_x h_y."""
    W, Np = geom.W, geom.Np
    up, vp, _ = geom.scaled(uvw)
    r0, nux = first_tap(up, W)
    s0, nuy = first_tap(vp, W)
    cx, cy = lm.weights(nux), lm.weights(nuy)
    tb = _bins(geom, uvw)
    V = np.asarray(vis, dtype=np.complex128)
    nm1 = geom.pixel_z() * geom.nscale                          # n - 1 on the image
    idx = _crop_index(geom)
    acc = np.zeros((geom.N, geom.N), dtype=np.complex128)
    for t in range(geom.t_lo, geom.t_hi + 1):
        sel = np.nonzero(tb == t)[0]
        if not sel.size:
            continue
        G = np.zeros((Np, Np), dtype=np.complex128)
        for b in range(W):                                      # step 3a: 2-D gridding
            rows = (s0[sel] + b) % Np
            for a in range(W):
                np.add.at(G, (rows, (r0[sel] + a) % Np), V[sel] * cy[sel, b] * cx[sel, a])
        P = np.fft.ifft2(G) * (Np * Np)                         # step 3b
        turns = (t / geom.nscale) * nm1                         # w[t] (n - 1)
        acc += P[np.ix_(idx, idx)] * np.exp(2j * np.pi * (turns - np.rint(turns)))  # 3c, 4
    hx = lm.h(geom.pixel_x())
    return (hx[None, :] * hx[:, None]) * acc                   # step 5: 2-D correction


def degrid_original(geom: Geometry, lm: LeastMisfit, image, uvw):
    """Algorithm 4: per w-bin correction, exp(-2 pi i w[t] (n - 1)), zero pad, FFT and
    2-D degridding of the bin's visibilities (the adjoint of grid_original)."""
    W, Np = geom.W, geom.Np
    up, vp, _ = geom.scaled(uvw)
    r0, nux = first_tap(up, W)
    s0, nuy = first_tap(vp, W)
    cx, cy = lm.weights(nux), lm.weights(nuy)
    tb = _bins(geom, uvw)
    hx = lm.h(geom.pixel_x())
    corrected = (hx[None, :] * hx[:, None]) * np.asarray(image, dtype=np.complex128)
    nm1 = geom.pixel_z() * geom.nscale
    idx = _crop_index(geom)
    out = np.zeros(r0.shape, dtype=np.complex128)
    for t in range(geom.t_lo, geom.t_hi + 1):
        sel = np.nonzero(tb == t)[0]
        if not sel.size:
            continue
        turns = (t / geom.nscale) * nm1
        Q = np.zeros((Np, Np), dtype=np.complex128)
        Q[np.ix_(idx, idx)] = corrected * np.exp(-2j * np.pi * (turns - np.rint(turns)))  # step 2a
        F = np.fft.fft2(Q)                                      # step 2b
        acc = np.zeros(sel.size, dtype=np.complex128)
        for b in range(W):                                      # step 2c: 2-D degridding
            rows = (s0[sel] + b) % Np
            for a in range(W):
                acc += F[rows, (r0[sel] + a) % Np] * (cx[sel, a] * cy[sel, b])
        out[sel] = acc
    return out
