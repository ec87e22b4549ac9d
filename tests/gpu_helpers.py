"""Shared helpers for the GPU parity tests (inputs from synth, references from the oracle)."""
import math

import numpy as np

from oracle import dft, wstack
from oracle.geometry import make_geometry
from oracle.lmfit import least_misfit
from paper_2101_11172_gb300 import synth

# FP32 path against FP64 references: the method itself sits near sqrt(3) E
# (2.1e-7 at W = 7, x0 = 0.25); FP32 storage, FFT and accumulation add a few
# 1e-7.  The bar is the stated target, 2e-6 relative RMS, for both the
# element-wise comparison with the FP64 oracle and with the exact DFT.
REL_TOL = 2e-6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


# Element-wise bar, in units of the reference's RMS: FP32 rounding spreads a
# near-Gaussian error of roughly equal size over every output, so |error| is
# close to Rayleigh distributed and its largest value over n outputs sits near
# sqrt(2 ln n) times its RMS -- 5.7 for n = 1e7, the largest count compared.
# With the RMS error allowed up to tol, no single output may be off by more
# than K_ELEM tol rms(ref).  A faint region that is wrong by more than that
# fails, however small the region.
K_ELEM = 6.0


def worst_element(a, ref):
    """(index, |a - ref| / rms(ref)) of the output farthest from the reference."""
    a, ref = np.asarray(a).ravel(), np.asarray(ref).ravel()
    err = np.abs(a - ref)
    i = int(np.argmax(err))
    return i, float(err[i] / np.sqrt(np.mean(np.abs(ref) ** 2)))


def assert_elementwise(a, ref, tol, what):
    """Every output within K_ELEM x tol x rms(ref) of the reference (prints the worst)."""
    i, e = worst_element(a, ref)
    print(f"{what}: worst element {i}: |error| = {e:.2e} rms(ref) (bar {K_ELEM * tol:.2e})")
    assert e <= K_ELEM * tol, (what, i, e, K_ELEM * tol)


def tol_for(W, x0):
    """Relative-RMS bar: 2e-6, or the method's own sqrt(3) E when that is larger."""
    return max(REL_TOL, 1.5 * math.sqrt(3) * least_misfit(W, x0).E)


def case(N=64, M=2000, W=7, fov=0.4, wfac=16.0, seed=7, x0=0.25):
    rng = synth.rng_for(0, 1000 + seed)
    R = 0.45 * N / fov
    uvw = synth.disc_uvw(M, R, 0.05 * R * wfac, rng)
    image = synth.point_sky(N, max(4, N // 4), rng) + 0.1 * synth.complex_normal(N * N, rng).reshape(N, N)
    vis = synth.complex_normal(M, rng)
    return dict(N=N, M=M, W=W, fov=fov, x0=x0, uvw=uvw, image=image, vis=vis,
                w_min=float(uvw[:, 2].min()), w_max=float(uvw[:, 2].max()))


def oracle_pair(c, z_offset=True):
    g = make_geometry(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], z_offset)
    lm = least_misfit(c["W"], g.x0)
    return g, lm, wstack.degrid(g, lm, c["image"], c["uvw"]), wstack.grid(g, lm, c["uvw"], c["vis"])


def dft_pair(c, g):
    lmn = dft.pixel_lmn(g)
    return dft.dft_degrid(c["uvw"], lmn, c["image"]), dft.dft_grid(c["uvw"], c["vis"], lmn).reshape(g.N, g.N)
