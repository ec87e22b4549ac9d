"""The survey-scale workload itself, through the C ABI, against the exact DFT.

N = 2048 (N' = 4096, x0 = 0.25), W = 7, l and m in +-0.25, 9,987,840
visibilities from 256 antennas on 8 h tracks: 370 w-planes, held as one
chunk of 376 planes (48 GB) on the compile-time 4096-point transforms with
TMA row copies.  This is the configuration the benchmark times.  The exact
operator (Eq. fourier_visibility and its adjoint) is evaluated by brute force
on 10^4 sampled visibilities and 1,024 sampled pixels with the oracle's
OpenMP C loops on every host core, and every sampled output must lie within
the element-wise bar as well as the 2e-6 relative-RMS target.
"""
import time

import numpy as np
import pytest

from gpu_helpers import REL_TOL, assert_elementwise, rel
from oracle import dft
from oracle.geometry import make_geometry
from paper_2101_11172_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_VIS = 10_000
N_PIX = 1024


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def test_survey_workload_against_dft(dev):
    from paper_2101_11172_gb300 import _lib
    from paper_2101_11172_gb300.wstack import Plan
    wl = synth.survey()
    assert wl.M == 9_987_840 and wl.N == 2048
    g = make_geometry(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range)
    with Plan(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range, device=dev) as p:
        assert (p.Np, p.Nw, p.t_lo) == (g.Np, g.Nw, g.t_lo) == (4096, 370, g.t_lo)
        assert p.planes_per_chunk >= p.Nw, "the survey runs as one plane chunk"
        uvw = torch.from_numpy(wl.uvw).to(dev)
        img = torch.from_numpy(wl.image.astype(np.complex64)).to(dev)
        vis = torch.from_numpy(wl.vis.astype(np.complex64)).to(dev)
        v = p.degrid(img, uvw)
        assert p.last_status == _lib.WS_OK
        d = p.grid(uvw, vis)
        assert p.last_status == _lib.WS_OK
        torch.cuda.synchronize()
        v = v.cpu().numpy().astype(np.complex128)
        d = d.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(2101)
    kv = rng.choice(wl.M, N_VIS, replace=False)
    rows = rng.integers(0, wl.N, N_PIX)
    cols = rng.integers(0, wl.N, N_PIX)
    t0 = time.perf_counter()
    nz_rows, nz_cols = np.nonzero(wl.image)
    v_ref = dft.dft_degrid(wl.uvw[kv], dft.pixel_lmn(g, nz_rows, nz_cols), wl.image[nz_rows, nz_cols])
    d_ref = dft.dft_grid(wl.uvw, wl.vis, dft.pixel_lmn(g, rows, cols))
    t_dft = time.perf_counter() - t0
    ev, ed = rel(v[kv], v_ref), rel(d[rows, cols], d_ref)
    print(f"survey: {wl.M} visibilities, {g.Nw} planes; vs DFT on {N_VIS} vis / {N_PIX} px: "
          f"degrid {ev:.2e}, grid {ed:.2e} (DFT {t_dft:.1f} s)")
    assert ev < REL_TOL and ed < REL_TOL
    assert_elementwise(v[kv], v_ref, REL_TOL, "survey degrid vs DFT")
    assert_elementwise(d[rows, cols], d_ref, REL_TOL, "survey grid vs DFT")
