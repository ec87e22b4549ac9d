"""Reduced-cost setting at full size: 4096^2 image, 5600^2 grid (mixed radix), W = 5, 5x10^7 visibilities.

The w-stack (282 planes of 5600^2, 71 GB) would fit the device; the test
caps the plan's workspace at 20 GB so that the plan works through it in
four chunks and footprints straddle chunk borders at full size.  The oracle's exact DFT checks sampled
outputs: 10^4 visibilities of the degridded point-source sky and 64 pixels
of the dirty image of all 5x10^7 visibilities.  The bar is the method's own
error, 1.5 sqrt(3) E(W = 5, x0 = 0.366) = 8e-4 relative RMS.
"""
import numpy as np
import pytest

from gpu_helpers import rel, tol_for
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


def test_reduced_cost_sampled_against_dft(dev, monkeypatch):
    from paper_2101_11172_gb300.wstack import Plan
    monkeypatch.setenv("WS_STACK_BYTES", str(20 * 10 ** 9))
    wl = synth.reduced_cost()
    geom = make_geometry(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range)
    rng = synth.rng_for(2, 9)
    with Plan(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range, device=dev) as p:
        assert (p.Np, p.Nw, p.t_lo) == (geom.Np, geom.Nw, geom.t_lo) and p.Np == 5600
        assert p.planes_per_chunk < p.Nw          # the stack is processed in chunks
        uvw = torch.from_numpy(wl.uvw).to(dev)
        v = p.degrid(torch.from_numpy(wl.image).to(torch.complex64).to(dev), uvw)
        st_v = p.last_status
        d = p.grid(uvw, torch.from_numpy(wl.vis).to(dev))
        st_d = p.last_status
        torch.cuda.synchronize()
        assert st_v == 0 and st_d == 0
        k = rng.choice(wl.M, size=10_000, replace=False)
        v_gpu = v[torch.from_numpy(k).to(dev)].cpu().numpy().astype(np.complex128)
        pix = rng.choice(wl.N * wl.N, size=64, replace=False)
        d_gpu = d.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy().astype(np.complex128)
        chunks = -(-p.Nw // p.planes_per_chunk)
    rows, cols = np.nonzero(wl.image)
    v_ref = dft.dft_degrid(wl.uvw[k], dft.pixel_lmn(geom, rows, cols), wl.image[rows, cols])
    d_ref = dft.dft_grid(wl.uvw, wl.vis, dft.pixel_lmn(geom, pix // wl.N, pix % wl.N))
    tol = tol_for(wl.W, geom.x0)
    ev, ed = rel(v_gpu, v_ref), rel(d_gpu, d_ref)
    print(f"reduced cost: N'={geom.Np}, {geom.Nw} planes in {chunks} chunks; "
          f"degrid {ev:.3e}, grid {ed:.3e} (bar {tol:.1e})")
    assert ev < tol and ed < tol
