"""Autograd wiring of DegridFunction, checked on the CPU with a dense stand-in plan.

The stand-in applies an explicit matrix A (degrid) and A^H (grid) in float64;
the checks are that autograd's gradient of chi^2 is 2 Re(A^H (A f - V)) /
sigma^2 for a real image, the conjugate-Wirtinger gradient 2 A^H (A f - V) /
sigma^2 for a complex one, and torch.autograd.gradcheck on both.  The CUDA
plan is exercised by the GPU tests; this file needs no device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2101_11172_gb300.autograd import chi2, degrid  # noqa: E402


class DensePlan:
    """degrid(f) = A vec(f), grid(V) = reshape(A^H V): an exact adjoint pair."""

    def __init__(self, A: torch.Tensor, N: int):
        self.A, self.N = A, N

    def degrid(self, image, uvw):
        return self.A @ image.reshape(-1)

    def grid(self, uvw, vis):
        return (self.A.conj().T @ vis).reshape(self.N, self.N)


def problem(seed=0, N=4, M=23):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, N * N, dtype=torch.complex128, generator=g)
    target = torch.randn(M, dtype=torch.complex128, generator=g)
    uvw = torch.zeros(M, 3, dtype=torch.float64)
    return DensePlan(A, N), A, target, uvw, g


def test_real_image_gradient_is_real_part_of_adjoint():
    plan, A, target, uvw, g = problem()
    f = torch.randn(4, 4, dtype=torch.float64, generator=g, requires_grad=True)
    sigma = 0.3
    loss = chi2(plan, f, uvw, target, sigma)
    loss.backward()
    r = A @ f.detach().reshape(-1).to(torch.complex128) - target
    want = (2 * (A.conj().T @ r).real / sigma ** 2).reshape(4, 4)
    assert f.grad.dtype == torch.float64
    assert torch.allclose(f.grad, want, rtol=1e-12, atol=1e-12)
    assert abs(loss.item() - (r.abs() ** 2).sum().item() / sigma ** 2) < 1e-9 * loss.item()


def test_complex_image_gradient_is_conjugate_wirtinger():
    plan, A, target, uvw, g = problem(1)
    f = torch.randn(4, 4, dtype=torch.complex128, generator=g, requires_grad=True)
    loss = chi2(plan, f, uvw, target, 1.0)
    loss.backward()
    r = A @ f.detach().reshape(-1) - target
    want = (2 * (A.conj().T @ r)).reshape(4, 4)
    assert torch.allclose(f.grad, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_gradcheck(dtype):
    plan, A, target, uvw, g = problem(2, N=3, M=7)
    f = torch.randn(3, 3, dtype=dtype, generator=g, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: degrid(plan, x, uvw), (f,))
    assert torch.autograd.gradcheck(lambda x: chi2(plan, x, uvw, target, 0.5), (f,))


def test_descent_reduces_chi2():
    """One steepest-descent step with an exact line search lowers chi^2 (a quadratic)."""
    plan, A, target, uvw, g = problem(3)
    f = torch.zeros(4, 4, dtype=torch.float64, requires_grad=True)
    loss0 = chi2(plan, f, uvw, target, 1.0)
    loss0.backward()
    d = -f.grad
    Ad = A @ d.reshape(-1).to(torch.complex128)
    r = A @ f.detach().reshape(-1).to(torch.complex128) - target
    step = -(torch.vdot(Ad, r).real / torch.vdot(Ad, Ad).real).item()
    loss1 = chi2(plan, (f.detach() + step * d), uvw, target, 1.0)
    assert step > 0 and loss1.item() < loss0.item()
