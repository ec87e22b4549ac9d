"""Least-squares imaging through the CUDA operators: conjugate gradients on chi^2
for the paper's 34-source sky (Appendix A, the field of Sections 6.3 and 7) drive
chi^2 down monotonically to the noise level and recover the sources.  The data
are exact (the oracle's DFT) plus noise."""
import json
import os

import numpy as np
import pytest

from oracle import dft
from oracle.geometry import make_geometry
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


def appendix_sky(N):
    """The Appendix A sources on an N x N map of the same 6-degree field: table
    pixel (X, Y) from the centre, 24 arcseconds each, lands on image pixel
    (N/2 + round(Y N / 900), N/2 + round(X N / 900)), row along m, column along l."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "appendix_a_sky.json")) as f:
        table = json.load(f)
    sky = np.zeros((N, N))
    scale = N / table["map_pixels"]
    for _, X, Y, flux in table["sources"]:
        sky[N // 2 + int(round(Y * scale)), N // 2 + int(round(X * scale))] += flux
    fov = np.deg2rad(table["field_deg"])
    return sky, fov


def test_cg_recovers_the_appendix_sky(dev):
    from paper_2101_11172_gb300.reconstruct import cg_image
    from paper_2101_11172_gb300.wstack import Plan
    N, M, sigma = 128, 60000, 0.01
    sky, fov = appendix_sky(N)
    assert np.count_nonzero(sky) == 34 and sky.sum() == 52.0
    rng = synth.rng_for(0, 3000)
    R = 0.45 * N / fov
    uvw = synth.disc_uvw(M, R, 0.05 * R * 20, rng)
    g = make_geometry(N, 0.25, 7, fov, float(uvw[:, 2].min()), float(uvw[:, 2].max()))
    rows, cols = np.nonzero(sky)
    vis = dft.dft_degrid(uvw, dft.pixel_lmn(g, rows, cols), sky[rows, cols]) + synth.complex_normal(M, rng, sigma)
    with Plan(N, 0.25, 7, fov, *g_range(uvw), device=dev) as p:
        f, hist = cg_image(p, torch.from_numpy(uvw).to(dev), torch.from_numpy(vis.astype(np.complex64)).to(dev),
                           sigma, iters=300)
        f = f.cpu().numpy().astype(np.float64)
    print("chi^2 / M by iteration:", [round(h / M, 3) for h in hist[::15]])
    assert all(b <= a * (1 + 1e-6) for a, b in zip(hist, hist[1:]))      # CG never raises chi^2 here
    # towards the noise level (about 1 - N^2 / (2 M) = 0.86 once every pixel is fitted): the
    # last modes, the unsampled corners of the uv plane, converge slowly, so 300 steps end
    # near it (chi^2 / M was 1.87 after 150)
    assert hist[-1] / M < 1.5 and hist[0] / hist[-1] > 1e5
    # the sources come back.  The visibilities fill a disc of 0.9 of the uv plane's width, so
    # the corners' Fourier modes stay unconstrained and the image is the sky seen through that
    # disc: the sky's own disc-limited image correlates with it at 0.79 and has 30 source
    # pixels among its 34 brightest.
    assert np.corrcoef(f.ravel(), sky.ravel())[0, 1] > 0.75
    top = set(np.argsort(f.ravel())[-34:])
    assert len(top & set(np.flatnonzero(sky))) >= 28


def g_range(uvw):
    return float(uvw[:, 2].min()), float(uvw[:, 2].max())
