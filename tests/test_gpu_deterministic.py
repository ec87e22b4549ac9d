"""Bit-for-bit reproducible gridding (WS_FLAG_DETERMINISTIC): the dirty image does
not depend on the order of the visibilities, nor on the order the binning's atomics
and the warps give them; it agrees with the default mode to FP32 rounding and with
the oracle at the usual bar.  Degridding is deterministic in every mode."""
import numpy as np
import pytest

from gpu_helpers import assert_elementwise, case, oracle_pair, rel, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def _grid(p, uvw, vis, dev):
    d = p.grid(torch.from_numpy(uvw).to(dev), torch.from_numpy(vis).to(torch.complex64).to(dev))
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("N", [128, 256])
def test_dirty_image_independent_of_visibility_order(dev, N):
    from paper_2101_11172_gb300 import WS_FLAG_DETERMINISTIC, _lib
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=N, M=8000, wfac=24.0, seed=89)
    perm = np.random.default_rng(5).permutation(c["M"])
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], flags=WS_FLAG_DETERMINISTIC,
              device=dev) as p:
        d1 = _grid(p, c["uvw"], c["vis"], dev)
        assert p.last_status == _lib.WS_OK
        d2 = _grid(p, c["uvw"], c["vis"], dev)
        d3 = _grid(p, np.ascontiguousarray(c["uvw"][perm]), np.ascontiguousarray(c["vis"][perm]), dev)
        assert np.array_equal(d1, d2) and np.array_equal(d1, d3)
        # degridding: the permuted call gives the permuted visibilities, bit for bit
        img = torch.from_numpy(c["image"]).to(torch.complex64).to(dev)
        v1 = p.degrid(img, torch.from_numpy(c["uvw"]).to(dev)).cpu().numpy()
        v3 = p.degrid(img, torch.from_numpy(np.ascontiguousarray(c["uvw"][perm])).to(dev)).cpu().numpy()
        assert np.array_equal(v1[perm], v3)
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as q:
        d0 = _grid(q, c["uvw"], c["vis"], dev)
    assert rel(d1, d0) < 1e-6
    g, lm, _, d_ref = oracle_pair(c)
    tol = tol_for(c["W"], g.x0)
    d1 = d1.astype(np.complex128)
    assert rel(d1, d_ref) < tol
    assert_elementwise(d1, d_ref, tol, f"deterministic grid, N = {N}")


def test_deterministic_across_plane_chunks_and_wide_footprints(dev, monkeypatch):
    # W = 10: a footprint reaches 3 t-tiles, so a plane chunk also takes the
    # bins of the two t-tiles before it (only their planes inside the chunk)
    from paper_2101_11172_gb300 import WS_FLAG_DETERMINISTIC, _lib
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=64, M=4000, W=10, wfac=40.0, seed=97)
    perm = np.random.default_rng(7).permutation(c["M"])
    monkeypatch.setenv("WS_PLANES_PER_CHUNK", "8")
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], flags=WS_FLAG_DETERMINISTIC,
              device=dev) as p:
        assert p.planes_per_chunk == 8 and p.Nw > 24
        d1 = _grid(p, c["uvw"], c["vis"], dev)
        assert p.last_status == _lib.WS_OK
        d3 = _grid(p, np.ascontiguousarray(c["uvw"][perm]), np.ascontiguousarray(c["vis"][perm]), dev)
        assert np.array_equal(d1, d3)
    g, lm, _, d_ref = oracle_pair(c)
    tol = tol_for(c["W"], g.x0)
    d1 = d1.astype(np.complex128)
    assert rel(d1, d_ref) < tol, rel(d1, d_ref)
    assert_elementwise(d1, d_ref, tol, "deterministic grid, W = 10, 8-plane chunks")
