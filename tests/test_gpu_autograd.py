"""Differentiable degridding on the GPU: 1024^2 image, 2048^2 grid, W = 7, 2x10^6 visibilities.

chi^2 = sum_k |V_k(f) - V_t,k|^2 / sigma^2 with V(f) the CUDA degridder and
its gradient from the CUDA gridder (the adjoint).  The references:
  * the exact gradient 2 Re(A^H (A f - V_t)) / sigma^2 on a 64 x 64 crop, with
    A f and A^H r by the FP64 brute-force DFT of the oracle;
  * central differences of the CUDA chi^2 on 64 random pixels (chi^2 is
    quadratic in f, so the central difference has no truncation error and the
    step can be large enough to rise above FP32 rounding);
  * the plain, non-differentiable calls: the forward is ws_degrid bit for bit,
    the backward is ws_grid up to summation order (gridding accumulates with
    shared-memory atomics, whose order varies from call to call).
"""
import numpy as np
import pytest

from gpu_helpers import REL_TOL, rel
from oracle import dft
from oracle.geometry import make_geometry
from paper_2101_11172_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CROP = 64


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def problem(dev):
    """The workload, its target visibilities (rounded to complex64, as the GPU sees them)
    and the exact residual r = A f - V_t, all from the oracle's DFT (both skies are sparse)."""
    wl = synth.differentiable()
    geom = make_geometry(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range)

    def exact_vis(img):
        rows, cols = np.nonzero(img)
        return dft.dft_degrid(wl.uvw, dft.pixel_lmn(geom, rows, cols), img[rows, cols])

    target = (exact_vis(wl.image) + wl.vis).astype(np.complex64)
    model = exact_vis(wl.estimate)
    resid = model - target.astype(np.complex128)
    return wl, geom, target, model, resid


@pytest.fixture(scope="module")
def plan(dev, problem):
    from paper_2101_11172_gb300.wstack import Plan
    wl = problem[0]
    p = Plan(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range, device=dev)
    yield p
    p.close()


def gpu_loss_and_grad(plan, wl, target, dev):
    from paper_2101_11172_gb300.autograd import chi2
    f = torch.tensor(wl.estimate, dtype=torch.float32, device=dev, requires_grad=True)
    uvw = torch.from_numpy(wl.uvw).to(dev)
    loss = chi2(plan, f, uvw, torch.from_numpy(target).to(dev), wl.sigma)
    loss.backward()
    return loss.item(), f.grad.detach(), uvw


def test_chi2_gradient_against_dft_gradient(dev, problem, plan):
    wl, geom, target, model, resid = problem
    loss, grad, _ = gpu_loss_and_grad(plan, wl, target, dev)
    # the crop is centred on the brightest source of the estimate
    i, j = np.unravel_index(np.argmax(wl.estimate), wl.estimate.shape)
    i0 = int(np.clip(i - CROP // 2, 0, wl.N - CROP))
    j0 = int(np.clip(j - CROP // 2, 0, wl.N - CROP))
    ii, jj = np.meshgrid(np.arange(i0, i0 + CROP), np.arange(j0, j0 + CROP), indexing="ij")
    g_exact = 2.0 * dft.dft_grid(wl.uvw, resid, dft.pixel_lmn(geom, ii.ravel(), jj.ravel())).real / wl.sigma ** 2
    g_gpu = grad[i0:i0 + CROP, j0:j0 + CROP].cpu().numpy().astype(np.float64).ravel()
    chi2_exact = float(np.sum(np.abs(resid) ** 2)) / wl.sigma ** 2
    # The gradient is A^H applied to a residual that carries the degridding error:
    # g~ - g = (A~^H - A^H) r~ + A^H (A~ - A) f.  Each operator is within the
    # 2e-6 relative bar, and the second term is relative to |A f|, not to |r|.
    ratio = float(np.linalg.norm(model) / np.linalg.norm(resid))
    tol = REL_TOL * (1.0 + ratio)
    err = rel(g_gpu, g_exact)
    print(f"chi2 {loss:.6e} exact {chi2_exact:.6e}; |Af|/|r| = {ratio:.2f}; grad rel err {err:.3e} (tol {tol:.2e})")
    assert abs(loss - chi2_exact) < 2 * tol * chi2_exact
    assert err < tol


def test_chi2_gradient_central_differences(dev, problem, plan):
    from paper_2101_11172_gb300.autograd import chi2
    wl, geom, target, model, resid = problem
    _, grad, uvw = gpu_loss_and_grad(plan, wl, target, dev)
    tgt = torch.from_numpy(target).to(dev)
    pix = synth.rng_for(3, 6).choice(wl.N * wl.N, size=64, replace=False)
    h = 0.1
    f = torch.tensor(wl.estimate, dtype=torch.float32, device=dev)
    fd = []
    with torch.no_grad():
        for p in pix:
            i, j = divmod(int(p), wl.N)
            fp, fm = f.clone(), f.clone()
            fp[i, j] += h
            fm[i, j] -= h
            fd.append((chi2(plan, fp, uvw, tgt, wl.sigma).item() - chi2(plan, fm, uvw, tgt, wl.sigma).item()) / (2 * h))
    fd = np.array(fd)
    g = grad.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy().astype(np.float64)
    err = np.abs(fd - g).max() / np.sqrt(np.mean(g ** 2))
    print(f"central differences: max |fd - grad| / rms(grad) = {err:.3e}")
    # chi^2 ~ 2e6 terms summed in FP64 from FP32 visibilities; its rounding noise
    # divided by 2h stays below 1e-4 of the gradient's scale
    assert err < 1e-3


def test_autograd_matches_plain_calls(dev, problem, plan):
    from paper_2101_11172_gb300.autograd import degrid
    wl, geom, target, model, resid = problem
    uvw = torch.from_numpy(wl.uvw).to(dev)
    f = torch.tensor(wl.estimate, dtype=torch.float32, device=dev, requires_grad=True)
    v = degrid(plan, f, uvw)
    gv = torch.from_numpy(synth.complex_normal(wl.M, synth.rng_for(3, 7)).astype(np.complex64)).to(dev)
    v.backward(gv)
    v_plain = plan.degrid(f.detach().to(torch.complex64), uvw)
    g_plain = plan.grid(uvw, gv)
    torch.cuda.synchronize()
    assert torch.equal(v.detach(), v_plain)
    g_auto = f.grad.double().cpu().numpy()
    g_ref = g_plain.real.double().cpu().numpy()
    assert rel(g_auto, g_ref) < 1e-6, rel(g_auto, g_ref)
    # and the forward is within the bar of the exact visibilities
    assert rel(v.detach().cpu().numpy().astype(np.complex128), model) < REL_TOL
