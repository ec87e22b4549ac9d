"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- no gridding, transform or
correction arithmetic -- so both the CUDA path and the FP64 oracle can be fed
from it.  The paper's own data (VLA B-array at 74 MHz with a 34-source sky,
Section 6.3; G55.7+3.4 and GMRT AMI001, Section 7) are not available, so these
stand-ins reproduce their shape: earth-rotation uvw tracks of a non-coplanar
array with a significant w range, and point-source skies.

Every generator takes a seed and uses numpy's PCG64; a workload is seeded
with ``SEED_BASE + index`` (index 0 = tiny, 1 = survey, 2 = reduced cost,
3 = differentiable, 4 = batched).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2101111720


def rng_for(index: int, stream: int = 0) -> np.random.Generator:
    """Independent sub-stream ``stream`` of workload ``index``."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE + index, stream])))


def complex_normal(n: int, rng: np.random.Generator, sigma: float = 1.0) -> np.ndarray:
    """CN(0, sigma^2): real and imaginary parts N(0, sigma^2/2)."""
    s = sigma / math.sqrt(2.0)
    return (rng.normal(0.0, s, n) + 1j * rng.normal(0.0, s, n)).astype(np.complex128)


def point_sky(N: int, n_src: int, rng: np.random.Generator, lo=0.1, hi=1.0) -> np.ndarray:
    """N x N image (rows = m, columns = l) with n_src unit-pixel sources at distinct pixels."""
    img = np.zeros((N, N), dtype=np.complex128)
    pos = rng.choice(N * N, size=n_src, replace=False)
    img.ravel()[pos] = rng.uniform(lo, hi, n_src)
    return img


def blob_sky(N: int, n_points: int, n_blobs: int, rng: np.random.Generator) -> np.ndarray:
    """Point sources plus circular Gaussian blobs (sigma 2-8 pixels)."""
    img = point_sky(N, n_points, rng)
    yy = np.arange(N)
    for _ in range(n_blobs):
        cy, cx = rng.uniform(0, N, 2)
        sig = rng.uniform(2.0, 8.0)
        amp = rng.uniform(0.1, 1.0)
        r = int(math.ceil(5 * sig))
        ys = yy[max(0, int(cy) - r): min(N, int(cy) + r + 1)]
        xs = yy[max(0, int(cx) - r): min(N, int(cx) + r + 1)]
        g = np.exp(-0.5 * (((ys[:, None] - cy) ** 2 + (xs[None, :] - cx) ** 2) / sig ** 2))
        img[ys[0]:ys[-1] + 1, xs[0]:xs[-1] + 1] += amp * g
    return img


def disc_uvw(M: int, radius: float, w_half: float, rng: np.random.Generator) -> np.ndarray:
    """(u, v) uniform in a disc of the given radius, w uniform in [-w_half, w_half]."""
    r = radius * np.sqrt(rng.uniform(0.0, 1.0, M))
    th = rng.uniform(0.0, 2 * math.pi, M)
    w = rng.uniform(-w_half, w_half, M)
    return np.stack([r * np.cos(th), r * np.sin(th), w], 1)


def array_uvw(n_ant: int, diameter_m: float, lat_deg: float, dec_deg: float,
              ha_hours: tuple, n_times: int, uv_max: float,
              rng: np.random.Generator) -> np.ndarray:
    """Earth-rotation tracks of a flat random array, scaled to max |(u,v)| = uv_max.

    Antennas are uniform in a disc of the given diameter on the local
    horizontal plane; baselines go local (east, north, up) -> equatorial
    (X, Y, Z) -> (u, v, w) at each hour angle, the textbook interferometer
    geometry.  The wavelength is chosen afterwards so that the longest
    projected (u, v) equals ``uv_max`` wavelengths.  Rows are time-major.
    """
    rad = 0.5 * diameter_m * np.sqrt(rng.uniform(0.0, 1.0, n_ant))
    th = rng.uniform(0.0, 2 * math.pi, n_ant)
    east, north = rad * np.cos(th), rad * np.sin(th)
    up = np.zeros(n_ant)
    lat = math.radians(lat_deg)
    X = -north * math.sin(lat) + up * math.cos(lat)
    Y = east
    Z = north * math.cos(lat) + up * math.sin(lat)
    ia, ib = np.triu_indices(n_ant, k=1)
    B = np.stack([X[ib] - X[ia], Y[ib] - Y[ia], Z[ib] - Z[ia]], 1)       # (nbl, 3) metres
    H = np.radians(15.0 * np.linspace(ha_hours[0], ha_hours[1], n_times))
    d = math.radians(dec_deg)
    sH, cH = np.sin(H)[:, None], np.cos(H)[:, None]
    Bx, By, Bz = B[None, :, 0], B[None, :, 1], B[None, :, 2]
    u = sH * Bx + cH * By
    v = -math.sin(d) * cH * Bx + math.sin(d) * sH * By + math.cos(d) * Bz
    w = math.cos(d) * cH * Bx - math.cos(d) * sH * By + math.sin(d) * Bz
    uvw = np.stack([u.ravel(), v.ravel(), w.ravel()], 1)
    scale = uv_max / np.sqrt(uvw[:, 0] ** 2 + uvw[:, 1] ** 2).max()
    return uvw * scale


@dataclass
class Workload:
    name: str
    N: int
    x0: float
    W: int
    fov: float
    uvw: np.ndarray
    image: np.ndarray = field(repr=False)
    vis: np.ndarray = field(repr=False)

    @property
    def M(self) -> int:
        return self.uvw.shape[0]

    @property
    def w_range(self):
        return float(self.uvw[:, 2].min()), float(self.uvw[:, 2].max())


def tiny(variant: str = "A", N: int = 256, M: int = 10_000, fov: float = 0.2,
         n_src: int = 50, W: int = 7, x0: float = 0.25) -> Workload:
    """Plain method, tiny: N = 256 from a 512 grid, l, m in +-0.1 rad, 10^4 visibilities.

    (u, v) uniform in a disc of radius R = 0.45 N / fov wavelengths; w uniform
    in +-0.05 R N (variant "A", several hundred w-planes) or +-0.05 R
    (variant "B", about ten planes); 50 point sources with amplitudes
    U(0.1, 1) for degridding; CN(0, 1) visibilities for gridding.
    """
    R = 0.45 * N / fov
    w_half = 0.05 * R * (N if variant == "A" else 1.0)
    uvw = disc_uvw(M, R, w_half, rng_for(0, 1 if variant == "A" else 11))
    image = point_sky(N, n_src, rng_for(0, 2))
    vis = complex_normal(M, rng_for(0, 3))
    return Workload(f"tiny-{variant}", N, x0, W, fov, uvw, image, vis)


def survey(N: int = 2048, n_ant: int = 256, n_times: int = 306, fov: float = 0.5,
           W: int = 7, x0: float = 0.25, sigma: float = 0.01, index: int = 1,
           ha_hours=(-4.0, 4.0)) -> Workload:
    """Survey-scale plain method: 256 antennas in a 10 km disc, 8 h tracks at dec -30.

    32,640 baselines x 306 times = 9,987,840 visibilities; latitude -30 deg
    (unstated in the workload, a reading); max |(u,v)| = 0.45 N / fov; sky of
    500 points plus 20 Gaussian blobs; visibilities to grid are CN(0, 1) plus
    CN(0, sigma^2) noise, stored as complex64.
    """
    uvw = array_uvw(n_ant, 10_000.0, -30.0, -30.0, ha_hours, n_times,
                    0.45 * N / fov, rng_for(index, 1))
    image = blob_sky(N, 500, 20, rng_for(index, 2))
    M = uvw.shape[0]
    vis = complex_normal(M, rng_for(index, 3)) + complex_normal(M, rng_for(index, 4), sigma)
    return Workload(f"survey-N{N}-M{M}", N, x0, W, fov, uvw, image, vis)


def survey_slab(w_half: float = 35.0, **kw) -> Workload:
    """The survey workload restricted to |w| < w_half: same image, grid and
    array, about 1.8 million visibilities on 17 w-planes (a small
    case for profiling the per-plane kernels)."""
    wl = survey(**kw)
    sel = abs(wl.uvw[:, 2]) < w_half
    return Workload(f"survey-slab-N{wl.N}-w{w_half:g}", wl.N, wl.x0, wl.W, wl.fov, wl.uvw[sel], wl.image,
                    wl.vis[sel])


@dataclass
class Chi2Workload(Workload):
    """A chi^2 imaging problem: ``image`` is the true (real) sky, ``vis`` the
    noise added to its visibilities, ``estimate`` the (real) image at which
    chi^2 and its gradient are evaluated."""
    sigma: float = 0.01
    estimate: np.ndarray = field(default=None, repr=False)


def differentiable(N: int = 1024, n_ant: int = 256, n_times: int = 61, fov: float = 0.5, W: int = 7,
                   x0: float = 0.25, sigma: float = 0.01, n_src: int = 200, index: int = 3) -> Chi2Workload:
    """Differentiable-imaging workload: chi^2 between degridded and target visibilities.

    Image 1024 x 1024 (grid 2048), the survey array (256 antennas in a 10 km
    disc, dec -30, 8 h) sampled 61 times: 32,640 x 61 = 1,991,040
    visibilities, max |(u,v)| = 0.45 N / fov.  True sky: 200 point sources
    with amplitudes U(0.1, 1); target noise CN(0, sigma^2).  The estimate is
    the true sky with each amplitude scaled by U(0.7, 1.3) plus 20 spurious
    sources with amplitudes U(0.05, 0.3).  Both images are real.
    """
    uvw = array_uvw(n_ant, 10_000.0, -30.0, -30.0, (-4.0, 4.0), n_times, 0.45 * N / fov, rng_for(index, 1))
    sky = point_sky(N, n_src, rng_for(index, 2)).real.copy()
    noise = complex_normal(uvw.shape[0], rng_for(index, 4), sigma)
    r = rng_for(index, 5)
    rows, cols = np.nonzero(sky)
    est = np.zeros_like(sky)
    est[rows, cols] = sky[rows, cols] * r.uniform(0.7, 1.3, rows.size)
    est += point_sky(N, 20, r, 0.05, 0.3).real
    return Chi2Workload(f"chi2-N{N}-M{uvw.shape[0]}", N, x0, W, fov, uvw, sky, noise, sigma=sigma, estimate=est)


def reduced_cost(N: int = 4096, n_ant: int = 256, n_times: int = 1532, fov: float = 0.5, W: int = 5,
                 x0: float = 0.375, sigma: float = 0.01, n_src: int = 500, index: int = 2) -> Workload:
    """Reduced-cost setting: image 4096 x 4096 from a 5600 x 5600 grid, W = 5.

    The survey array (256 antennas in a 10 km disc, dec -30) tracked for 4 h
    (hour angles -2 .. +2) with 1532 samples: 32,640 x 1532 = 50,004,480
    visibilities, max |(u,v)| = 0.45 N / fov.  x0 = 0.375 is the reading of
    the setting's grid sizes (about 5461 padded, which the 7-smooth rule
    makes 5600).  Sky: 500 point sources U(0.1, 1) (sparse, so the exact
    visibilities are cheap); visibilities to grid are CN(0, 1) plus
    CN(0, sigma^2) noise, stored as complex64.
    """
    uvw = array_uvw(n_ant, 10_000.0, -30.0, -30.0, (-2.0, 2.0), n_times, 0.45 * N / fov, rng_for(index, 1))
    image = point_sky(N, n_src, rng_for(index, 2))
    M = uvw.shape[0]
    vis = (complex_normal(M, rng_for(index, 3)) + complex_normal(M, rng_for(index, 4), sigma)).astype(np.complex64)
    return Workload(f"reduced-cost-N{N}-M{M}", N, x0, W, fov, uvw, image, vis)


def batched(n: int = 64, sizes=(512, 1024, 2048), m_range=(1e4, 5e6), W: int = 7, x0: float = 0.25,
            index: int = 4) -> list:
    """Serving-style batch: n independent instances, each with its own seeded array and sky.

    Instance i draws from sub-stream 100 + i: image side uniform over
    ``sizes``; a target visibility count log-uniform in ``m_range``; an
    array of n_ant antennas (at most what the count allows, at most 256) in
    a 10 km disc at latitude -30; declination U(-70, 10) degrees; a track of
    U(1, 8) hours centred on hour angle U(-2, 2); field of view U(0.2, 0.5)
    rad; max |(u,v)| = 0.45 N / fov; n_src ~ U{20..200} point sources with
    amplitudes U(0.1, 1); visibilities to grid CN(0, 1) as complex64.
    M = baselines x times is the target rounded to whole time samples.
    """
    out = []
    for i in range(n):
        rng = rng_for(index, 100 + i)
        N = int(rng.choice(sizes))
        m_target = float(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]))))
        ant_max = int((1 + math.sqrt(1 + 8 * m_target)) / 2)
        n_ant = int(rng.integers(min(16, ant_max), min(256, ant_max) + 1))
        nbl = n_ant * (n_ant - 1) // 2
        n_times = max(1, int(round(m_target / nbl)))
        dec = float(rng.uniform(-70.0, 10.0))
        span, centre = float(rng.uniform(1.0, 8.0)), float(rng.uniform(-2.0, 2.0))
        fov = float(rng.uniform(0.2, 0.5))
        uvw = array_uvw(n_ant, 10_000.0, -30.0, dec, (centre - span / 2, centre + span / 2), n_times,
                        0.45 * N / fov, rng)
        image = point_sky(N, int(rng.integers(20, 201)), rng)
        vis = complex_normal(uvw.shape[0], rng).astype(np.complex64)
        out.append(Workload(f"batch{i}-N{N}-M{uvw.shape[0]}", N, x0, W, fov, uvw, image, vis))
    return out
