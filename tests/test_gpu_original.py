"""The original W-stacking (Algorithms 3 and 4) on the GPU, against the oracle's
Algorithms 3 and 4 and against the exact DFT, beside the improved method on the
same data (Section 6.2: the binning error falls only as 1 / N_w)."""
import math

import numpy as np
import pytest

from gpu_helpers import REL_TOL, rel
from oracle import dft, wstack
from oracle.geometry import make_geometry, make_geometry_original
from oracle.lmfit import least_misfit
from paper_2101_11172_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def problem():
    N, fov, M = 64, 0.4, 2000
    rng = synth.rng_for(0, 2000)
    R = 0.45 * N / fov
    uvw = synth.disc_uvw(M, R, 0.05 * R * 30, rng)
    img = synth.point_sky(N, 12, rng)
    vis = synth.complex_normal(M, rng)
    return dict(N=N, fov=fov, M=M, uvw=uvw, img=img, vis=vis, w=(float(uvw[:, 2].min()), float(uvw[:, 2].max())))


def run(p, dev, bins, flags=0):
    from paper_2101_11172_gb300.wstack import Plan
    with Plan(p["N"], 0.25, 7, p["fov"], *p["w"], flags=flags, device=dev, original_bins=bins) as plan:
        uvw = torch.from_numpy(p["uvw"]).to(dev)
        v = plan.degrid(torch.from_numpy(p["img"]).to(torch.complex64).to(dev), uvw)
        st = plan.last_status
        d = plan.grid(uvw, torch.from_numpy(p["vis"]).to(torch.complex64).to(dev))
        torch.cuda.synchronize()
        assert (st, plan.last_status) == (0, 0)
        return (v.cpu().numpy().astype(np.complex128), d.cpu().numpy().astype(np.complex128), plan.nscale, plan.n0)


def test_original_matches_oracle_algorithms_3_and_4(dev, problem):
    p = problem
    lm = least_misfit(7, 0.25)
    for bins in (20, 80):
        v, d, nscale, n0 = run(p, dev, bins)
        g = make_geometry_original(p["N"], 0.25, 7, p["fov"], *p["w"], bins)
        assert math.isclose(nscale, g.nscale, rel_tol=1e-12) and n0 == 1.0
        v_ref = wstack.degrid_original(g, lm, p["img"], p["uvw"])
        d_ref = wstack.grid_original(g, lm, p["uvw"], p["vis"])
        # FP32 against FP64 of the same approximation
        assert rel(v, v_ref) < REL_TOL and rel(d, d_ref) < REL_TOL, (bins, rel(v, v_ref), rel(d, d_ref))


def test_original_error_against_dft_falls_as_one_over_bins(dev, problem):
    p = problem
    g0 = make_geometry(p["N"], 0.25, 7, p["fov"], *p["w"])
    lmn = dft.pixel_lmn(g0)
    v_dft = dft.dft_degrid(p["uvw"], lmn, p["img"])
    d_dft = dft.dft_grid(p["uvw"], p["vis"], lmn).reshape(p["N"], p["N"])
    errs = []
    for bins in (20, 40, 80):
        v, d, _, _ = run(p, dev, bins)
        errs.append((rel(v, v_dft), rel(d, d_dft)))
    for (a, b), (c, e) in zip(errs, errs[1:]):
        assert 1.8 < a / c < 2.2 and 1.7 < b / e < 2.3, errs
    v, d, _, _ = run(p, dev, 0)                  # the improved method on the same data
    improved = max(rel(v, v_dft), rel(d, d_dft))
    print("original, 20/40/80 bins:", errs, " improved:", improved)
    assert improved < REL_TOL and errs[-1][0] > 1e4 * improved


def test_original_rejects_too_few_bins_and_even_width(dev, problem):
    from paper_2101_11172_gb300 import WsError
    from paper_2101_11172_gb300.wstack import Plan
    p = problem
    with pytest.raises(WsError):
        Plan(p["N"], 0.25, 7, p["fov"], *p["w"], device=dev, original_bins=1)
    with pytest.raises(WsError):
        Plan(p["N"], 0.25, 6, p["fov"], *p["w"], device=dev, original_bins=40)
