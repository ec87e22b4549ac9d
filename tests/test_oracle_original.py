"""Pins of the oracle's original W-stacking (Algorithms 3 and 4).

* With every w on a bin centre there is no binning error: what is left is the
  two-dimensional least-misfit error, sqrt(2) E(W, x0) (Section 3.3 applied to
  two axes).
* Otherwise a visibility in bin t is computed as if measured at w[t]: a phase
  error 2 pi (w - w[t]) (n - 1) with w - w[t] uniform over a bin of width dw.
  To first order the relative RMS error of a point-source sky is
  2 pi (dw / sqrt 12) sqrt(sum a^2 (n - 1)^2 / sum a^2), and it halves each
  time the number of bins doubles (Section 6.2: the error goes as 1 / N_w).
* Algorithms 3 and 4 are adjoint.
"""
import math

import numpy as np
import pytest

from oracle import dft, wstack
from oracle.geometry import make_geometry_original, n_minus_one
from oracle.lmfit import least_misfit
from paper_2101_11172_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def problem():
    N, fov, M = 64, 0.4, 2000
    rng = synth.rng_for(0, 2000)
    R = 0.45 * N / fov
    uvw = synth.disc_uvw(M, R, 0.05 * R * 30, rng)
    img = synth.point_sky(N, 12, rng)
    vis = synth.complex_normal(M, rng)
    return dict(N=N, fov=fov, uvw=uvw, img=img, vis=vis, lm=least_misfit(7, 0.25),
                w=(float(uvw[:, 2].min()), float(uvw[:, 2].max())))


def test_on_bin_centres_only_the_2d_gridding_error_remains(problem):
    p = problem
    g = make_geometry_original(p["N"], 0.25, 7, p["fov"], *p["w"], 40)
    uvw = p["uvw"].copy()
    uvw[:, 2] = np.round(uvw[:, 2] * g.nscale) / g.nscale
    lmn = dft.pixel_lmn(g)
    e2 = math.sqrt(2) * p["lm"].E
    ev = rel(wstack.degrid_original(g, p["lm"], p["img"], uvw), dft.dft_degrid(uvw, lmn, p["img"]))
    ed = rel(wstack.grid_original(g, p["lm"], uvw, p["vis"]),
             dft.dft_grid(uvw, p["vis"], lmn).reshape(p["N"], p["N"]))
    assert 0.2 * e2 < ev < 1.5 * e2 and 0.2 * e2 < ed < 1.5 * e2, (ev, ed, e2)


def test_binning_error_matches_first_order_and_halves_with_twice_the_bins(problem):
    p = problem
    errs = []
    for Nw in (20, 40, 80):
        g = make_geometry_original(p["N"], 0.25, 7, p["fov"], *p["w"], Nw)
        v = wstack.degrid_original(g, p["lm"], p["img"], p["uvw"])
        err = rel(v, dft.dft_degrid(p["uvw"], dft.pixel_lmn(g), p["img"]))
        rows, cols = np.nonzero(p["img"])
        a = np.abs(p["img"][rows, cols])
        l = g.pixel_lm()
        nm1 = n_minus_one(l[cols], l[rows])
        pred = 2 * math.pi / (g.nscale * math.sqrt(12)) * math.sqrt(np.sum(a ** 2 * nm1 ** 2) / np.sum(a ** 2))
        assert abs(err / pred - 1) < 0.05, (Nw, err, pred)
        errs.append(err)
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs


def test_algorithms_3_and_4_are_adjoint(problem):
    p = problem
    g = make_geometry_original(p["N"], 0.25, 7, p["fov"], *p["w"], 30)
    v = wstack.degrid_original(g, p["lm"], p["img"], p["uvw"])
    d = wstack.grid_original(g, p["lm"], p["uvw"], p["vis"])
    lhs, rhs = np.vdot(v, p["vis"]), np.vdot(p["img"], d)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_bins_follow_the_width():
    g = make_geometry_original(64, 0.25, 7, 0.4, -100.0, 100.0, 50)
    assert g.nscale == 0.25 and (g.t_lo, g.t_hi) == (-25, 25) and g.n0 == 1.0
