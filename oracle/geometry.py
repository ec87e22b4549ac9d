"""Normalised coordinates and plan sizes of the improved W-stacking method, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 3.3 (the "Making a map" box: ``u' = u / du`` with
``du = 1/(N' dl)``, ``x = l/(N' dl)``), Section 5.1 (normalised image
coordinates, ``x = x0 l / l_max``), Section 5.2 (``w' = n_scale w`` and the
pre-phase ``exp(-2 pi i w (n0 - 1))``), Eq. z-on-sphere, Eq. n_params /
n_params_no_offset and Eq. N_{w'}+W of Section 5.3, and Eq. N_w of Section 4.

Readings where the paper leaves a choice:

* The FFT size ``N'`` is the smallest multiple of 32 with no prime factor
  above 7 that is at least ``N/(2 x0)``; the cropping parameter actually used
  is ``x0_eff = N/(2 N')`` and ``z0 = x0_eff`` (Section 6 recommends
  ``x0 = y0 = z0``).
* Pixel ``j`` of an ``N``-pixel axis, ``j = -N/2 .. N/2-1``, sits at
  ``l_j = j * dl`` with ``dl = fov/N`` and ``l_max = fov/2``.
* ``n_min`` is taken at the map corner ``l = m = l_max`` (Section 5.1), so
  every pixel has ``z`` in ``[-z0, z0]``.
* The planes used are exactly those the data can touch: with the tap rule of
  Section 3.3 (``first = floor(w' + W/2) - W + 1``), ``t_lo`` is the first tap
  of ``w'_min`` and ``t_hi`` the last tap of ``w'_max``.  Eq. N_{w'}+W gives
  the count bound ``N_w' > dn dw/(2 z0) + W`` that this never exceeds by more
  than one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _seven_smooth(n: int) -> bool:
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def fft_size(N: int, x0: float) -> int:
    """Smallest multiple of 32, 7-smooth, that is >= N/(2 x0)."""
    need = N / (2.0 * x0)
    n = 32 * max(1, math.ceil(need / 32.0 - 1e-12))
    while not _seven_smooth(n):
        n += 32
    return n


def n_minus_one(l, m):
    """n - 1 = sqrt(1 - l^2 - m^2) - 1 without cancellation."""
    r2 = np.asarray(l, dtype=np.float64) ** 2 + np.asarray(m, dtype=np.float64) ** 2
    return -r2 / (1.0 + np.sqrt(1.0 - r2))


def n_params(lmax: float, mmax: float, z0: float, z_offset: bool = True):
    """(n_scale, n0): Eq. n_params (z-offset) or Eq. n_params_no_offset."""
    one_minus_nmin = -float(n_minus_one(lmax, mmax))
    if z_offset:
        nscale = one_minus_nmin / (2.0 * z0)
        n0 = 1.0 - z0 * nscale
    else:
        nscale = one_minus_nmin / z0
        n0 = 1.0
    return nscale, n0


def layers_improved(dn: float, dw: float, z0: float, W: int, z_offset: bool = True) -> int:
    """Smallest integer strictly above the bound of Eq. N_{w'}+W (or its no-offset form)."""
    bound = dn * dw / ((2.0 if z_offset else 1.0) * z0) + W
    return int(math.floor(bound)) + 1


def layers_original(dn: float, dw: float) -> int:
    """Smallest integer satisfying Eq. N_w: N_w >= 2 pi (n_max - n_min)(w_max - w_min)."""
    return int(math.ceil(2.0 * math.pi * dn * dw - 1e-9))


def first_tap(coord, W: int):
    """Integer index of the first of the W grid points a coordinate touches, and nu.

    Section 3.3: the taps of ``u'`` are ``r = floor(u' + W/2) - W + 1 + i``,
    ``i = 0..W-1``, and ``nu = u' + (W-1)/2 - floor(u' + W/2)`` lies in
    ``[-1/2, 1/2)``; tap i then carries ``C(s_i - nu)``, ``s_i = i - (W-1)/2``.
    """
    c = np.asarray(coord, dtype=np.float64)
    fl = np.floor(c + 0.5 * W)
    return (fl - W + 1).astype(np.int64), c + 0.5 * (W - 1) - fl


@dataclass(frozen=True)
class Geometry:
    N: int
    Np: int
    x0: float          # effective cropping parameter N/(2 N'); also y0 and z0
    W: int
    fov: float
    nscale: float
    n0: float
    t_lo: int
    t_hi: int
    z_offset: bool = True

    @property
    def dl(self) -> float:
        return self.fov / self.N

    @property
    def lmax(self) -> float:
        return 0.5 * self.fov

    @property
    def Nw(self) -> int:
        return self.t_hi - self.t_lo + 1

    def pixel_lm(self):
        """l_j (= m_j) for j = -N/2 .. N/2-1."""
        return (np.arange(self.N) - self.N // 2) * self.dl

    def pixel_x(self):
        """Normalised x_j = j / N' (Section 3.3 box, step 2)."""
        return (np.arange(self.N) - self.N // 2) / self.Np

    def pixel_z(self):
        """z(x, y) of Eq. z-on-sphere on the N x N image, indexed [i (m), j (l)]."""
        l = self.pixel_lm()
        nm1 = n_minus_one(l[None, :], l[:, None])
        return (nm1 + (1.0 - self.n0)) / self.nscale

    def scaled(self, uvw):
        """(u', v', w') = (l_max u / x0, m_max v / y0, n_scale w) (Section 5.2)."""
        uvw = np.asarray(uvw, dtype=np.float64)
        k = self.lmax / self.x0
        return uvw[:, 0] * k, uvw[:, 1] * k, uvw[:, 2] * self.nscale


def make_geometry(N: int, x0: float, W: int, fov: float, w_min: float, w_max: float,
                  z_offset: bool = True) -> Geometry:
    if N <= 0 or N % 2:
        raise ValueError("N must be positive and even")
    Np = fft_size(N, x0)
    x0e = N / (2.0 * Np)
    lmax = 0.5 * fov
    nscale, n0 = n_params(lmax, lmax, x0e, z_offset)
    t_lo = int(first_tap(nscale * w_min, W)[0])
    t_hi = int(first_tap(nscale * w_max, W)[0]) + W - 1
    return Geometry(N=N, Np=Np, x0=x0e, W=W, fov=fov, nscale=nscale, n0=n0,
                    t_lo=t_lo, t_hi=t_hi, z_offset=z_offset)


def make_geometry_original(N: int, x0: float, W: int, fov: float, w_min: float, w_max: float,
                           Nw: int) -> Geometry:
    """Original W-stacking (Algorithms 3 and 4): Nw w-bins of width (w_max - w_min)/Nw.

    The bins are centred on multiples of the bin width (w' = w n_scale with
    n_scale = Nw / (w_max - w_min) rounded to the nearest integer), a shift of
    the lattice of Algorithm 3's centres w_min + (t + 1/2) dw that leaves the
    nearest-bin rule and the spacing unchanged.  The phase of bin t is
    exp(2 pi i w[t] (n - 1)), so n0 = 1 and z = (n - 1) / n_scale.  W is the
    width of the two-dimensional (u, v) kernel.
    """
    if N <= 0 or N % 2 or Nw < 1 or not w_max > w_min:
        raise ValueError("need even N > 0, Nw >= 1 and w_max > w_min")
    Np = fft_size(N, x0)
    nscale = Nw / (w_max - w_min)
    t_lo = int(math.floor(nscale * w_min + 0.5))
    t_hi = int(math.floor(nscale * w_max + 0.5))
    return Geometry(N=N, Np=Np, x0=N / (2.0 * Np), W=W, fov=fov, nscale=nscale, n0=1.0,
                    t_lo=t_lo, t_hi=t_hi, z_offset=False)
