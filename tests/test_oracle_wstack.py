"""Pins of the FP64 Algorithms 1, 2, 5, 6 and of the brute-force DFT."""
import math

import numpy as np
import pytest

from oracle import dft, wstack
from oracle.geometry import first_tap, make_geometry, n_minus_one
from oracle.lmfit import least_misfit
from paper_2101_11172_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# -- the exact operator --------------------------------------------------------

def test_dft_c_matches_numpy_transcription():
    g = make_geometry(16, 0.25, 7, 0.3, -60, 60)
    rng = np.random.default_rng(5)
    uvw = rng.uniform(-40, 40, (20, 3))
    f = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    V = synth.complex_normal(20, rng)
    lmn = dft.pixel_lmn(g)
    assert rel(dft.dft_degrid(uvw, lmn, f), dft.dft_degrid_numpy(uvw, lmn, f)) < 1e-14
    assert rel(dft.dft_grid(uvw, V, lmn), dft.dft_grid_numpy(uvw, V, lmn)) < 1e-14


def test_dft_closed_forms():
    # One unit point source at pixel (i0, j0): V_k = exp(-2 pi i (u l + v m + w (n - 1))).
    g = make_geometry(32, 0.25, 7, 0.4, -100, 100)
    rng = np.random.default_rng(6)
    uvw = rng.uniform(-80, 80, (50, 3))
    f = np.zeros((32, 32), complex)
    f[3, 29] = 1.0
    l, m = g.pixel_lm()[29], g.pixel_lm()[3]
    want = np.exp(-2j * np.pi * (uvw[:, 0] * l + uvw[:, 1] * m + uvw[:, 2] * n_minus_one(l, m)))
    got = dft.dft_degrid(uvw, dft.pixel_lmn(g), f)
    assert np.abs(got - want).max() < 1e-12
    # One visibility V = 1 at (u, v, w): d = exp(+2 pi i (...)); d at the map centre is 1.
    d = dft.dft_grid(uvw[:1], np.ones(1), dft.pixel_lmn(g)).reshape(32, 32)
    assert abs(d[16, 16] - 1) < 1e-14 and np.allclose(np.abs(d), 1, atol=1e-13)


# -- one dimension: Algorithms 1 and 2 ------------------------------------------

@pytest.mark.parametrize("W", [4, 7])
def test_1d_algorithms_against_dft(W):
    N, Np = 64, 128
    lm = least_misfit(W, 0.25)
    rng = np.random.default_rng(W)
    up = rng.uniform(-60, 60, 400)
    V = synth.complex_normal(400, rng)
    x = (np.arange(N) - N // 2) / Np
    exact_d = np.exp(2j * np.pi * np.outer(x, up)) @ V
    assert rel(wstack.grid_1d(lm, Np, N, up, V), exact_d) < 1.5 * lm.E
    f = rng.normal(size=N) + 1j * rng.normal(size=N)
    exact_v = np.exp(-2j * np.pi * np.outer(up, x)) @ f
    assert rel(wstack.degrid_1d(lm, Np, f, up), exact_v) < 1.5 * lm.E
    # Algorithm 2 is the adjoint of Algorithm 1 (Section 3.2)
    lhs = np.vdot(wstack.degrid_1d(lm, Np, f, up), V)
    rhs = np.vdot(f, wstack.grid_1d(lm, Np, N, up, V))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


# -- three dimensions: Algorithms 5 and 6 ---------------------------------------

def small_case(N=32, M=300, W=7, wfac=8.0, fov=0.4, seed=1):
    rng = np.random.default_rng(seed)
    R = 0.45 * N / fov
    uvw = synth.disc_uvw(M, R, 0.05 * R * wfac, rng)
    g = make_geometry(N, 0.25, W, fov, uvw[:, 2].min(), uvw[:, 2].max())
    lm = least_misfit(W, g.x0)
    img = synth.point_sky(N, 10, rng) + 0.3 * rng.normal(size=(N, N))
    V = synth.complex_normal(M, rng)
    return g, lm, uvw, img, V


@pytest.mark.parametrize("W,wfac", [(7, 1.0), (7, 8.0), (5, 4.0), (4, 4.0)])
def test_3d_against_dft_within_sqrt3_E(W, wfac):
    # Section 6.3 / Figure 8: the 3-D error stays near sqrt(3) E (quadrature sum
    # of three 1-D errors).  A dropped term, a wrong sign or a swapped axis gives
    # an error of order one.
    g, lm, uvw, img, V = small_case(W=W, wfac=wfac, N=48 if W == 7 else 64, M=400)
    lmn = dft.pixel_lmn(g)
    bound = math.sqrt(3) * lm.E
    eg = rel(wstack.grid(g, lm, uvw, V), dft.dft_grid(uvw, V, lmn).reshape(g.N, g.N))
    ed = rel(wstack.degrid(g, lm, img, uvw), dft.dft_degrid(uvw, lmn, img))
    assert eg < 1.5 * bound and ed < 1.5 * bound, (eg, ed, bound)
    assert eg > 0.2 * bound and ed > 0.2 * bound                # the method's error, not luck


def test_3d_adjoint_identity(golden):
    # <degrid(f), V> = <f, grid(V)> (Section 3.2; the MemTrq check of Section 7
    # passed at a few 1e-10, the FP64 oracle must do far better).
    g, lm, uvw, img, V = small_case(W=7, wfac=8.0)
    lhs = np.vdot(wstack.degrid(g, lm, img, uvw), V)
    rhs = np.vdot(img, wstack.grid(g, lm, uvw, V))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert 1e-12 < golden["adjoint_consistency"]["value"]


def test_dropping_hz_ruins_accuracy():
    # Section 6.3: the full 3-D correction h_x h_y h_z is essential.
    g, lm, uvw, img, V = small_case(W=7, wfac=8.0)
    exact = dft.dft_grid(uvw, V, dft.pixel_lmn(g)).reshape(g.N, g.N)
    good = rel(wstack.grid(g, lm, uvw, V), exact)
    bad = rel(wstack.grid(g, lm, uvw, V, with_hz=False), exact)
    assert bad > 1e4 * good


def test_planar_array_reduces_to_2d():
    # Section 6.3: with all w = 0 the problem is 2-D mapping.  The 3-D result
    # must agree with plain 2-D least-misfit gridding (Algorithm 1 in x and y)
    # to within the z-direction error alone.
    g0, lm, uvw, img, V = small_case(W=7, wfac=0.0)
    uvw = uvw.copy()
    uvw[:, 2] = 0.0
    g = make_geometry(g0.N, 0.25, 7, g0.fov, 0.0, 0.0)
    d3 = wstack.grid(g, lm, uvw, V)
    up, vp, _ = g.scaled(uvw)
    r0, nux = first_tap(up, 7)
    s0, nuy = first_tap(vp, 7)
    cx, cy = lm.weights(nux), lm.weights(nuy)
    G = np.zeros((g.Np, g.Np), complex)
    for b in range(7):
        for a in range(7):
            np.add.at(G, ((s0 + b) % g.Np, (r0 + a) % g.Np), V * cx[:, a] * cy[:, b])
    idx = (np.arange(g.N) - g.N // 2) % g.Np
    hx = lm.h(g.pixel_x())
    d2 = (hx[:, None] * hx[None, :]) * (np.fft.ifft2(G) * g.Np ** 2)[np.ix_(idx, idx)]
    assert rel(d3, d2) < 1.5 * lm.E


@pytest.mark.slow
def test_tiny_workload_B_against_dft():
    # The tiny workload (N = 256, 10^4 visibilities, ~10 planes) end to end.
    wl = synth.tiny("B")
    g = make_geometry(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range)
    lm = least_misfit(wl.W, g.x0)
    lmn = dft.pixel_lmn(g)
    bound = math.sqrt(3) * lm.E
    assert rel(wstack.grid(g, lm, wl.uvw, wl.vis),
               dft.dft_grid(wl.uvw, wl.vis, lmn).reshape(wl.N, wl.N)) < 1.5 * bound
    assert rel(wstack.degrid(g, lm, wl.image, wl.uvw), dft.dft_degrid(wl.uvw, lmn, wl.image)) < 1.5 * bound
