"""Image reconstruction on top of the gridder/degridder (Section 7's use).

The paper uses its operators inside an iterative imager (its Section 7 runs
them as the forward and adjoint operators of a maximum-entropy code).  This
module gives the plain least-squares counterpart: conjugate gradients on the
normal equations of

    chi^2(f) = sum_k |(A f)_k - V_k|^2 / sigma^2 + lam |f|^2,

i.e. (A^H A + lam sigma^2) f = A^H V, with A = ws_degrid and A^H = ws_grid of
one plan.  Images are real (a real sky) unless ``real=False``.  Vector
algebra runs in PyTorch on the device; every application of A and A^H is
the CUDA library's.
"""
from __future__ import annotations

import torch

from .wstack import Plan


def _apply_normal(plan: Plan, f: torch.Tensor, uvw: torch.Tensor, lam_s2: float, real: bool) -> torch.Tensor:
    img = torch.complex(f, torch.zeros_like(f)) if real else f
    g = plan.grid(uvw, plan.degrid(img.contiguous(), uvw))
    g = g.real if real else g
    return g + lam_s2 * f


def _dot(a: torch.Tensor, b: torch.Tensor) -> float:
    return float(torch.vdot(a.reshape(-1).to(torch.complex128), b.reshape(-1).to(torch.complex128)).real)


def chi2(plan: Plan, f: torch.Tensor, uvw: torch.Tensor, vis: torch.Tensor, sigma: float, real: bool = True) -> float:
    img = torch.complex(f, torch.zeros_like(f)) if real else f
    r = plan.degrid(img.contiguous(), uvw) - vis
    return float((r.real.double() ** 2 + r.imag.double() ** 2).sum()) / sigma ** 2


def cg_image(plan: Plan, uvw: torch.Tensor, vis: torch.Tensor, sigma: float, iters: int = 30, lam: float = 0.0,
             real: bool = True, f0: torch.Tensor | None = None, tol: float = 1e-8):
    """Least-squares image by conjugate gradients; returns (image, [chi^2 per iteration]).

    uvw is bound to the plan for the iterations (``Plan.bind``): the tap rule and
    the tile sort are made once, and every application of A and A^H reuses them."""
    N = plan.N
    plan.bind(uvw)
    dtype = torch.float32 if real else torch.complex64
    f = torch.zeros(N, N, dtype=dtype, device=vis.device) if f0 is None else f0.clone()
    b = plan.grid(uvw, vis)
    b = b.real if real else b
    r = b - _apply_normal(plan, f, uvw, lam * sigma ** 2, real)
    p = r.clone()
    rr = _dot(r, r)
    rr0 = rr
    history = [chi2(plan, f, uvw, vis, sigma, real)]
    for _ in range(iters):
        Ap = _apply_normal(plan, p, uvw, lam * sigma ** 2, real)
        alpha = rr / _dot(p, Ap)
        f = f + alpha * p
        r = r - alpha * Ap
        rr_new = _dot(r, r)
        history.append(chi2(plan, f, uvw, vis, sigma, real))
        if rr_new <= tol * tol * rr0:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return f, history
