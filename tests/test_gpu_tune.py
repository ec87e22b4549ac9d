"""Gridding tiles of 16, 32 and 64 rows (ws_plan_tune and its JSON cache): every
shape gives the oracle's answer, the tuner keeps the fastest on the caller's data
and records its timings, and plans made with WS_TUNE_CACHE set take the cached shape."""
import json

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


def _tensors(c, dev):
    return (torch.from_numpy(c["uvw"]).to(dev), torch.from_numpy(c["vis"]).to(torch.complex64).to(dev),
            torch.from_numpy(c["image"]).to(torch.complex64).to(dev))


def test_tuner_cache_and_every_tile_shape(dev, tmp_path, monkeypatch):
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=128, M=6000, wfac=24.0, seed=83)
    uvw, vis, img = _tensors(c, dev)
    cache = tmp_path / "tune.json"
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        assert p.tile_rows == 16
        rows = p.tune(uvw, vis, img, cache_path=str(cache))
        assert rows in (16, 32, 64) and p.tile_rows == rows
        data = json.loads(cache.read_text())
        (key, entry), = data.items()
        assert key.endswith(f"|N'={p.Np}|W={p.W}") and entry["tile_rows"] == rows
        assert set(entry["ms"]) == {"16", "32", "64"} and all(v > 0 for v in entry["ms"].values())
        assert entry["ms"][str(rows)] == min(entry["ms"].values())
        # a cached entry is applied without timing
        assert p.tune(uvw, vis, img, cache_path=str(cache)) == rows
    g, lm, v_ref, d_ref = oracle_pair(c)
    tol = tol_for(c["W"], g.x0)
    for forced in (16, 32, 64):
        data[key]["tile_rows"] = forced
        cache.write_text(json.dumps(data))
        monkeypatch.setenv("WS_TUNE_CACHE", str(cache))
        with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
            assert p.tile_rows == forced
            v = p.degrid(img, uvw).cpu().numpy().astype(np.complex128)
            d = p.grid(uvw, vis).cpu().numpy().astype(np.complex128)
            # a bound set on a re-tiled plan
            p.bind(uvw)
            vb = p.degrid(img, uvw).cpu().numpy().astype(np.complex128)
        assert rel(v, v_ref) < tol and rel(d, d_ref) < tol, (forced, rel(v, v_ref), rel(d, d_ref))
        assert_elementwise(v, v_ref, tol, f"degrid, {forced}-row tiles")
        assert_elementwise(d, d_ref, tol, f"grid, {forced}-row tiles")
        assert np.array_equal(vb, v)
        monkeypatch.delenv("WS_TUNE_CACHE")


def test_tile_rows_must_divide_the_grid(dev, tmp_path, monkeypatch):
    # N' = 160 (N = 80): 64-row tiles do not divide it; a cache entry asking for them is refused
    from paper_2101_11172_gb300 import _lib
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=80, M=1500, W=7, seed=17)
    uvw, vis, img = _tensors(c, dev)
    cache = tmp_path / "tune.json"
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        assert p.Np == 160
        rows = p.tune(uvw, vis, img, cache_path=str(cache))
        assert rows in (16, 32)
        data = json.loads(cache.read_text())
        (key, entry), = data.items()
        assert set(entry["ms"]) == {"16", "32"}
    data[key]["tile_rows"] = 64
    cache.write_text(json.dumps(data))
    monkeypatch.setenv("WS_TUNE_CACHE", str(cache))
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        assert p.tile_rows == 16                       # the invalid entry is ignored
        assert _lib.WS_OK == 0


def test_tiles_spanning_the_whole_grid(dev, tmp_path, monkeypatch):
    # N' = 32 with 32-row tiles: one tile holds every row of the grid, so the
    # footprints near its edge wrap around inside the tile (the gridding
    # kernel's two-span path, and a degridding bin that is a whole column)
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=16, M=1500, W=7, seed=29)
    uvw, vis, img = _tensors(c, dev)
    cache = tmp_path / "tune.json"
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        assert p.Np == 32
        p.tune(uvw, vis, img, cache_path=str(cache))
    data = json.loads(cache.read_text())
    (key, entry), = data.items()
    data[key]["tile_rows"] = 32
    cache.write_text(json.dumps(data))
    monkeypatch.setenv("WS_TUNE_CACHE", str(cache))
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        assert p.tile_rows == 32
        v = p.degrid(img, uvw).cpu().numpy().astype(np.complex128)
        d = p.grid(uvw, vis).cpu().numpy().astype(np.complex128)
    g, lm, v_ref, d_ref = oracle_pair(c)
    tol = tol_for(c["W"], g.x0)
    assert rel(v, v_ref) < tol and rel(d, d_ref) < tol, (rel(v, v_ref), rel(d, d_ref))
    assert_elementwise(v, v_ref, tol, "degrid, N' = 32, 32-row tiles")
    assert_elementwise(d, d_ref, tol, "grid, N' = 32, 32-row tiles")


def test_deterministic_plans_skip_tiles_whose_ring_does_not_fit(dev, tmp_path, monkeypatch):
    # deterministic gridding sums in 64-bit cells: at W = 7 a 64-row tile's ring
    # of planes would need about 250 KB of shared memory, so the tuner leaves that
    # shape out and a cache entry asking for it is ignored
    from paper_2101_11172_gb300 import WS_FLAG_DETERMINISTIC
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=128, M=4000, wfac=24.0, seed=31)
    uvw, vis, img = _tensors(c, dev)
    cache = tmp_path / "tune.json"
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], flags=WS_FLAG_DETERMINISTIC,
              device=dev) as p:
        rows = p.tune(uvw, vis, img, cache_path=str(cache))
        assert rows in (16, 32)
    data = json.loads(cache.read_text())
    (key, entry), = data.items()
    assert set(entry["ms"]) == {"16", "32"}
    data[key]["tile_rows"] = 64
    cache.write_text(json.dumps(data))
    monkeypatch.setenv("WS_TUNE_CACHE", str(cache))
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], flags=WS_FLAG_DETERMINISTIC,
              device=dev) as p:
        assert p.tile_rows == 16
        d = p.grid(uvw, vis).cpu().numpy().astype(np.complex128)
    g, lm, _, d_ref = oracle_pair(c)
    tol = tol_for(c["W"], g.x0)
    assert rel(d, d_ref) < tol
    assert_elementwise(d, d_ref, tol, "deterministic grid after an ignored 64-row cache entry")
