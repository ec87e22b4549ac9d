"""ws_degrid_noalloc (collected last): the allocation-free degridding entry point.

Callers that cannot allocate device memory while running use this entry
point; it must give what ws_degrid gives, through the C ABI, call after call,
with its scratch taken from the library's fixed device array.
"""
import numpy as np
import pytest

from gpu_helpers import REL_TOL, case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def test_noalloc_degrid_matches_degrid_twice(dev):
    from paper_2101_11172_gb300 import _lib
    c = case(N=128, M=3000, wfac=16.0, seed=41)
    with torch.cuda.device(dev):
        plan = _lib.ws_plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], 0)
        try:
            uvw = torch.from_numpy(c["uvw"]).to(dev)
            img = torch.from_numpy(c["image"]).to(torch.complex64).to(dev)
            ref = torch.empty(c["M"], dtype=torch.complex64, device=dev)
            out = torch.empty_like(ref)
            stream = torch.cuda.current_stream(dev).cuda_stream
            assert _lib.ws_degrid(plan, img.data_ptr(), uvw.data_ptr(), c["M"], ref.data_ptr(), stream) == 0
            want = ref.cpu().numpy()
            for _ in range(2):                     # the shared scratch keeps the previous call's contents
                out.fill_(float("nan"))
                st = _lib.ws_degrid_noalloc(plan, img.data_ptr(), uvw.data_ptr(), c["M"], out.data_ptr(), stream)
                assert st == _lib.WS_OK, _lib.ws_last_error()
                got = out.cpu().numpy()
                assert np.all(np.isfinite(got))
                assert rel(got, want) < REL_TOL
        finally:
            _lib.ws_destroy(plan)


def test_noalloc_rejects_problems_beyond_its_scratch(dev):
    from paper_2101_11172_gb300 import _lib
    with torch.cuda.device(dev):
        plan = _lib.ws_plan(2048, 0.25, 7, 0.5, -100.0, 100.0, 0)   # 8 planes of 4096^2 = 1 GiB > 64 MiB
        try:
            uvw = torch.zeros(4, 3, dtype=torch.float64, device=dev)
            img = torch.zeros(2048, 2048, dtype=torch.complex64, device=dev)
            out = torch.empty(4, dtype=torch.complex64, device=dev)
            with pytest.raises(_lib.WsError) as err:
                _lib.ws_degrid_noalloc(plan, img.data_ptr(), uvw.data_ptr(), 4, out.data_ptr(),
                                       torch.cuda.current_stream(dev).cuda_stream)
            assert err.value.status == _lib.WS_ERR_ARG and "64 MiB" in str(err.value)
        finally:
            _lib.ws_destroy(plan)


def _noalloc_against_degrid(dev, c, flags=0, calls=2):
    """ws_degrid_noalloc against ws_degrid on one plan, `calls` times in a row; returns the plan's
    planes per chunk of the regular path and the plane count."""
    from paper_2101_11172_gb300 import _lib
    with torch.cuda.device(dev):
        plan = _lib.ws_plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], flags)
        try:
            info = _lib.ws_plan_info(plan)
            uvw = torch.from_numpy(c["uvw"]).to(dev)
            img = torch.from_numpy(c["image"]).to(torch.complex64).to(dev)
            ref = torch.empty(c["M"], dtype=torch.complex64, device=dev)
            out = torch.empty_like(ref)
            stream = torch.cuda.current_stream(dev).cuda_stream
            assert _lib.ws_degrid(plan, img.data_ptr(), uvw.data_ptr(), c["M"], ref.data_ptr(), stream) == 0
            want = ref.cpu().numpy()
            for _ in range(calls):
                out.fill_(float("nan"))
                st = _lib.ws_degrid_noalloc(plan, img.data_ptr(), uvw.data_ptr(), c["M"], out.data_ptr(), stream)
                assert st == _lib.WS_OK, _lib.ws_last_error()
                got = out.cpu().numpy()
                assert np.all(np.isfinite(got))
                assert rel(got, want) < REL_TOL, rel(got, want)
            return info.Nw
        finally:
            _lib.ws_destroy(plan)


def test_noalloc_several_plane_chunks(dev):
    # N' = 256 (512 KiB per plane) with a w-range of about 210 planes: the fixed scratch
    # holds about 120 planes after the records and the image, so the allocation-free
    # path carves its own chunk size and adds the chunks' contributions in turn
    c = case(N=128, M=3000, wfac=170.0, seed=43)
    Nw = _noalloc_against_degrid(dev, c)
    assert Nw * 256 * 256 * 8 > (64 << 20), Nw


def test_noalloc_hermitian_folding(dev):
    # a real sky with w of both signs: visibilities at w < 0 are degridded at -(u, v, w)
    # and conjugated afterwards, in the allocation-free path as in ws_degrid
    from paper_2101_11172_gb300 import WS_FLAG_HERMITIAN
    c = case(N=128, M=3000, wfac=40.0, seed=47)
    c["image"] = c["image"].real.astype(np.complex128)
    assert (c["uvw"][:, 2] < 0).mean() > 0.3 and (c["uvw"][:, 2] > 0).mean() > 0.3
    _noalloc_against_degrid(dev, c, flags=WS_FLAG_HERMITIAN)
