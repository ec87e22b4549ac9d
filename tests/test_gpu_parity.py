"""CUDA path (through the C ABI) against the FP64 oracle and the exact DFT."""
import math
import os

import numpy as np
import pytest

from gpu_helpers import REL_TOL, assert_elementwise, case, dft_pair, oracle_pair, rel, tol_for
from oracle import dft, wstack
from oracle.geometry import make_geometry
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


def run_gpu(c, dev, flags=0):
    from paper_2101_11172_gb300.wstack import Plan
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], flags=flags, device=dev) as p:
        uvw = torch.from_numpy(c["uvw"]).to(dev)
        v = p.degrid(torch.from_numpy(c["image"]).to(torch.complex64).to(dev), uvw)
        st_v = p.last_status
        d = p.grid(uvw, torch.from_numpy(c["vis"]).to(torch.complex64).to(dev))
        st_d = p.last_status
        torch.cuda.synchronize()
        info = dict(Np=p.Np, Nw=p.Nw, t_lo=p.t_lo, n0=p.n0, nscale=p.nscale, x0=p.x0, E=p.error_bound,
                    P=p.planes_per_chunk, st=(st_v, st_d))
        return v.cpu().numpy().astype(np.complex128), d.cpu().numpy().astype(np.complex128), info


def check_against_oracle(c, dev, flags=0, z_offset=True):
    v, d, info = run_gpu(c, dev, flags)
    g, lm, v_ref, d_ref = oracle_pair(c, z_offset)
    assert (info["Np"], info["Nw"], info["t_lo"]) == (g.Np, g.Nw, g.t_lo)
    assert math.isclose(info["nscale"], g.nscale, rel_tol=1e-12) and math.isclose(info["n0"], g.n0, rel_tol=1e-14)
    assert math.isclose(info["E"], lm.E, rel_tol=1e-4)
    tol = tol_for(c["W"], g.x0)
    assert rel(v, v_ref) < tol, ("degrid", rel(v, v_ref), tol)
    assert rel(d, d_ref) < tol, ("grid", rel(d, d_ref), tol)
    # element-wise: no single output far off, measured against the RMS of the reference
    assert_elementwise(v, v_ref, tol, "degrid vs oracle")
    assert_elementwise(d, d_ref, tol, "grid vs oracle")
    return v, d, g, lm, v_ref, d_ref, info


@pytest.mark.parametrize("variant", ["B", "A"])
def test_tiny_workload_against_oracle_and_dft(dev, variant):
    wl = synth.tiny(variant)
    c = dict(N=wl.N, M=wl.M, W=wl.W, fov=wl.fov, x0=wl.x0, uvw=wl.uvw, image=wl.image, vis=wl.vis,
             w_min=wl.w_range[0], w_max=wl.w_range[1])
    v, d, g, lm, v_ref, d_ref, info = check_against_oracle(c, dev)
    v_dft, d_dft = dft_pair(c, g)
    assert rel(v, v_dft) < REL_TOL and rel(d, d_dft) < REL_TOL
    assert_elementwise(v, v_dft, REL_TOL, "degrid vs DFT")
    assert_elementwise(d, d_dft, REL_TOL, "grid vs DFT")
    print(f"tiny-{variant}: planes {g.Nw}; GPU vs DFT degrid {rel(v, v_dft):.2e} grid {rel(d, d_dft):.2e}; "
          f"GPU vs oracle {rel(v, v_ref):.2e} {rel(d, d_ref):.2e}")


@pytest.mark.parametrize("W", [4, 5, 7, 8])
def test_widths(dev, W):
    check_against_oracle(case(N=64, M=1500, W=W, seed=W), dev)


def test_nonstandard_grid_and_x0(dev):
    # N' = 384 (2^7 * 3) from N = 200, x0 = 0.3: effective x0 = 0.2604
    c = case(N=200, M=1500, W=6, x0=0.3, fov=0.3, seed=3)
    v, d, g, *_ = check_against_oracle(c, dev)
    assert g.Np == 384


def test_radix_ten_plan(dev):
    # N' = 160 = 2^5 5: the runtime plan pairs one 2 with the 5 (radices 16, 10)
    c = case(N=80, M=1500, W=7, seed=17)
    v, d, g, *_ = check_against_oracle(c, dev)
    assert g.Np == 160


def test_no_z_offset_variant(dev):
    from paper_2101_11172_gb300 import WS_FLAG_NO_Z_OFFSET
    check_against_oracle(case(seed=11), dev, flags=WS_FLAG_NO_Z_OFFSET, z_offset=False)


def test_plane_chunks_agree(dev, monkeypatch):
    c = case(N=64, M=3000, wfac=40.0, seed=5)
    v1, d1, i1 = run_gpu(c, dev)
    monkeypatch.setenv("WS_PLANES_PER_CHUNK", "8")
    v2, d2, i2 = run_gpu(c, dev)
    assert i1["P"] >= i1["Nw"] and i2["P"] == 8 and i2["Nw"] > 24
    assert rel(v2, v1) < 1e-6 and rel(d2, d1) < 1e-6
    g, lm, v_ref, d_ref = oracle_pair(c)
    assert rel(v2, v_ref) < REL_TOL and rel(d2, d_ref) < REL_TOL


@pytest.mark.parametrize("N", [256, 512])
def test_compile_time_plans_against_oracle(dev, N):
    # N' = 512 and 1024 run the compile-time FFT plans: TMA row copies in
    # inv_rows (first-stage butterflies for only 32 or 64 of the 256 threads),
    # the stepped screen in fwd_rows (several CTAs per row, 8-plane runs)
    c = case(N=N, M=3000, W=7, seed=21)
    v, d, g, *_ = check_against_oracle(c, dev)
    assert g.Np == 2 * N


def test_compile_time_plan_chunks_agree(dev, monkeypatch):
    # several chunks on a compile-time plan: TMA plane coordinates relative to
    # the chunk and the compensated sum carried between inv_rows launches
    c = case(N=256, M=3000, W=7, seed=22)
    v1, d1, i1 = run_gpu(c, dev)
    monkeypatch.setenv("WS_PLANES_PER_CHUNK", "8")
    v2, d2, i2 = run_gpu(c, dev)
    assert i1["Np"] == 512 and i1["P"] >= i1["Nw"] and i2["P"] == 8 and i2["Nw"] > 24
    assert rel(v2, v1) < 1e-6 and rel(d2, d1) < 1e-6
    g, lm, v_ref, d_ref = oracle_pair(c)
    assert rel(v2, v_ref) < REL_TOL and rel(d2, d_ref) < REL_TOL


def test_wraparound_at_grid_edge(dev):
    # u' within W/2 of +-N'/2: taps wrap onto the opposite edge; the periodic
    # inverse DFT keeps the result exact (compare with the DFT directly).
    c = case(N=64, M=600, seed=13)
    Np = make_geometry(64, 0.25, 7, c["fov"], c["w_min"], c["w_max"]).Np
    k = (Np / 2) / (Np * c["fov"] / 64)        # u' = N'/2  <->  u = k
    rng = np.random.default_rng(3)
    c["uvw"][:200, 0] = k * rng.uniform(0.985, 1.015, 200) * rng.choice([-1, 1], 200)
    c["uvw"][200:400, 1] = k * rng.uniform(0.985, 1.015, 200) * rng.choice([-1, 1], 200)
    v, d, g, lm, v_ref, d_ref, info = check_against_oracle(c, dev)
    v_dft, d_dft = dft_pair(c, g)
    assert rel(v, v_dft) < REL_TOL and rel(d, d_dft) < REL_TOL


def test_adjoint_identity(dev):
    # <degrid(f), V> = <f, grid(V)>: the GPU pair is adjoint up to FP32 rounding
    c = case(N=128, M=5000, seed=17)
    v, d, _ = run_gpu(c, dev)
    lhs = np.vdot(v, c["vis"])
    rhs = np.vdot(c["image"], d)
    assert abs(lhs - rhs) < 2e-6 * abs(lhs)


def test_hermitian_folding_real_sky(dev):
    # Section 5.4: for a real sky, w < 0 is handled as the conjugate visibility at
    # -(u, v, w); the folded plan needs planes for |w| only.  Degridding must still
    # give every visibility of the real sky, gridding the real dirty image.
    from paper_2101_11172_gb300 import WS_FLAG_HERMITIAN
    c = case(N=128, M=5000, wfac=40.0, seed=19)
    c["image"] = c["image"].real.astype(np.complex128)
    assert (c["uvw"][:, 2] < 0).mean() > 0.3 and (c["uvw"][:, 2] > 0).mean() > 0.3
    v, d, info = run_gpu(c, dev, flags=WS_FLAG_HERMITIAN)
    _, _, plain = run_gpu(c, dev)
    assert info["st"] == (0, 0)
    assert info["Nw"] < 0.6 * plain["Nw"]
    g = make_geometry(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"])
    v_dft, d_dft = dft_pair(c, g)
    tol = tol_for(c["W"], g.x0)
    assert rel(v, v_dft) < tol, rel(v, v_dft)
    assert np.all(d.imag == 0)
    assert rel(d.real, d_dft.real) < tol, rel(d.real, d_dft.real)
    # the folded pair is adjoint on real images: Re <degrid(f), V> = <f, grid(V)>
    lhs = np.vdot(v, c["vis"]).real
    rhs = float(np.sum(c["image"].real * d.real))
    assert abs(lhs - rhs) < 2e-6 * np.linalg.norm(v) * np.linalg.norm(c["vis"])


def test_divide_by_n_acts_on_the_sky_brightness(dev):
    # Section 5.2: f = I / n.  With WS_FLAG_DIVIDE_BY_N the calls take I and return the dirty
    # image divided by n: degrid(I) = plain degrid(I / n), grid(V) = plain grid(V) / n.
    from oracle.geometry import n_minus_one
    from paper_2101_11172_gb300 import WS_FLAG_DIVIDE_BY_N
    c = case(N=128, M=4000, fov=0.8, seed=29)
    g = make_geometry(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"])
    l = g.pixel_lm()
    n = 1.0 + n_minus_one(l[None, :], l[:, None])
    v1, d1, _ = run_gpu(c, dev, flags=WS_FLAG_DIVIDE_BY_N)
    c0 = dict(c, image=c["image"] / n)
    v0, d0, _ = run_gpu(c0, dev)
    assert rel(v1, v0) < 1e-6 and rel(d1, d0 / n) < 1e-6
    assert abs(np.vdot(v1, c["vis"]) - np.vdot(c["image"], d1)) < 2e-6 * abs(np.vdot(v1, c["vis"]))


def test_edge_counts_and_drops(dev):
    from paper_2101_11172_gb300 import _lib
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=64, M=1000, seed=19)
    uvw = c["uvw"].copy()
    uvw[0, 2] = c["w_max"] + 50.0            # beyond the plan's w-range
    uvw[1, 2] = c["w_min"] - 50.0
    uvw[2, 0] = np.nan
    with Plan(64, 0.25, 7, c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        tu = torch.from_numpy(uvw).to(dev)
        img = torch.from_numpy(c["image"]).to(torch.complex64).to(dev)
        v = p.degrid(img, tu)
        assert p.last_status == _lib.WS_ERR_UV_RANGE and p.dropped() == 3
        vv = v.cpu().numpy()
        assert np.all(vv[:3] == 0)
        # the others match a clean run over the same visibilities
        ok = torch.from_numpy(c["uvw"][3:]).to(dev)
        v_ok = p.degrid(img, ok)
        assert p.last_status == _lib.WS_OK
        assert np.array_equal(v_ok.cpu().numpy(), vv[3:]) or rel(vv[3:], v_ok.cpu().numpy()) < 1e-7
        d = p.grid(tu, torch.from_numpy(c["vis"]).to(torch.complex64).to(dev))
        assert p.last_status == _lib.WS_ERR_UV_RANGE and p.dropped() == 3
        # M = 0 and M = 1
        z = p.grid(tu[:0], torch.zeros(0, dtype=torch.complex64, device=dev))
        assert p.last_status == _lib.WS_OK and float(z.abs().max()) == 0.0
        e = p.degrid(img, tu[:0])
        assert e.numel() == 0 and p.last_status == _lib.WS_OK
        one = p.degrid(img, ok[:1])
        assert rel(one.cpu().numpy(), v_ok[:1].cpu().numpy()) < 1e-6
    # w exactly at the ends of the range is inside
    c2 = case(N=64, M=500, seed=23)
    c2["uvw"][0, 2], c2["uvw"][1, 2] = c2["w_min"], c2["w_max"]
    check_against_oracle(c2, dev)


def test_repeat_calls_deterministic_shapes(dev):
    # A plan reused across calls with growing M gives the same answers.
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=64, M=4000, seed=29)
    with Plan(64, 0.25, 7, c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        uvw = torch.from_numpy(c["uvw"]).to(dev)
        img = torch.from_numpy(c["image"]).to(torch.complex64).to(dev)
        a = p.degrid(img, uvw[:100]).cpu().numpy()
        b = p.degrid(img, uvw).cpu().numpy()
        c_ = p.degrid(img, uvw[:100]).cpu().numpy()
        assert rel(b[:100], a) < 1e-7 and rel(c_, a) < 1e-7
