"""Least-misfit gridding function C(u') and gridding correction h(x), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What the paper fixes (Section 3.3):

* Eq. csum2 -- the misfit of one visibility whose grid offset is nu:
  ``L(x, nu) = 1 - h(x) * sum_s C(s - nu) exp(2 pi i (s - nu) x)`` with
  ``s = -(W-1)/2 .. (W-1)/2`` and ``-1/2 <= nu < 1/2`` (the paper prints the
  upper limit as ``< -1/2``; it is read as ``< 1/2``).
* Eq. norm_bound -- the error bound
  ``E^2 = 1/(2 x0) * int_{-x0}^{x0} int_{-1/2}^{1/2} |L(x, nu)|^2 dnu dx`` and
  the map error ``l(x) = int |L(x, nu)|^2 dnu``.
* The least-misfit pair (C, h) is, for given W and x0, the even C supported on
  ``[-W/2, W/2]`` and the real h that minimise E (the "Making a map" box of
  Section 3.3; the construction itself is only cited there).

How this module computes the minimiser (the paper gives no algorithm):

* Write ``c_s(nu) = C(s - nu)`` for ``nu`` in ``[-1/2, 1/2]``.  For a fixed h,
  the best ``c(nu)`` solves a linear least-squares problem whose matrix does
  not depend on nu, so ``c_s(nu)`` is an entire function of nu; it is
  represented exactly enough by a Legendre series in ``2 nu`` of degree D.
  Evenness of C, ``C(u) = C(-u)``, is ``c_{-s}(nu) = c_s(-nu)`` and is built
  into the parameterisation.
* For fixed C the best h is pointwise in x:
  ``h(x) = int Re a(x,nu) dnu / int |a(x,nu)|^2 dnu`` with
  ``a(x, nu) = sum_s c_s(nu) exp(2 pi i (s - nu) x)``.  This defines h at any
  argument, which is how ``h_z(z(x, y))`` is evaluated off any grid (the paper
  interpolates a table instead, Section 5.3).
* With h eliminated this way, the misfit is a function of the Legendre
  coefficients alone, and its small residual makes Gauss-Newton converge in a
  handful of iterations.  (Plain alternation between the two partial
  minimisations converges to the same point but needs thousands of sweeps.)
  A Levenberg-Marquardt step replaces a Gauss-Newton step that fails to lower
  E, and for large x0 the minimiser is followed up from x0 = 1/4 (see
  ``least_misfit``).

Pins (tests/test_oracle_lmfit.py): E(W=7, x0=0.25) against the quoted
1.3e-7 (Section 6); the layer multipliers 6, 27, 500 quoted for Figure 3; the
top-hat closed form of Section 6; evenness; W=1 against the top hat; E
falling with W at every x0 up to 0.45 and W up to 14, and reaching FP64
rounding level at W = 14, x0 = 1/4 (Section 6.3: double precision at W = 14).
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as _leg


def gauss_legendre(n: int, a: float, b: float):
    """n-point Gauss-Legendre nodes and weights on [a, b]."""
    t, w = _leg.leggauss(n)
    return 0.5 * (b - a) * t + 0.5 * (b + a), 0.5 * (b - a) * w


def tap_offsets(W: int) -> np.ndarray:
    """The W values s = -(W-1)/2 .. (W-1)/2 of Eq. csum2 (half-integers for even W)."""
    return np.arange(W, dtype=np.float64) - 0.5 * (W - 1)


@dataclass(frozen=True)
class LeastMisfit:
    """A least-misfit pair for width ``W`` and cropping parameter ``x0``.

    ``beta[i, k]`` is the coefficient of the Legendre polynomial ``P_k(2 nu)``
    in ``c_i(nu) = C(s_i - nu)``, ``s_i = i - (W-1)/2``.
    """

    W: int
    x0: float
    beta: np.ndarray          # (W, D+1)
    E: float                  # error bound of Eq. norm_bound, fine quadrature
    n_nu: int = 96            # nu-quadrature used to define h off-grid

    @property
    def degree(self) -> int:
        return self.beta.shape[1] - 1

    def weights(self, nu) -> np.ndarray:
        """``c_i(nu)`` for every tap i: array of shape ``nu.shape + (W,)``."""
        nu = np.asarray(nu, dtype=np.float64)
        P = _leg.legvander(2.0 * nu, self.degree)          # (..., D+1)
        return P @ self.beta.T

    def h(self, x) -> np.ndarray:
        """Gridding correction at arbitrary x (the h-step formula above)."""
        x = np.asarray(x, dtype=np.float64)
        flat = x.reshape(-1)
        nq, wn = gauss_legendre(self.n_nu, -0.5, 0.5)
        c = self.weights(nq)                               # (nn, W)
        s = tap_offsets(self.W)
        out = np.empty_like(flat)
        step = 4096
        for a0 in range(0, flat.size, step):
            xs = flat[a0:a0 + step]
            ph = 2.0 * np.pi * (s[None, None, :] - nq[None, :, None]) * xs[:, None, None]
            a = (c[None, :, :] * np.exp(1j * ph)).sum(-1)    # (nx, nn)
            R = (wn[None, :] * a.real).sum(1)
            Q = (wn[None, :] * (a.real ** 2 + a.imag ** 2)).sum(1)
            out[a0:a0 + step] = R / Q
        return out.reshape(x.shape)


def interpolated_h(lm: "LeastMisfit", n_table: int = 4097, order: int = 10):
    """h on [-x0, x0] by the paper's own recipe (Section 5.3): a table of h on a
    uniform grid and polynomial interpolation of high degree within it.

    The table holds the exact h-step values at ``n_table`` uniform points; each
    argument is interpolated by the Lagrange polynomial through the ``order``
    table points nearest to it.  Returns a callable.
    """
    x0 = lm.x0
    xs = np.linspace(-x0, x0, n_table)
    hs = lm.h(xs)
    step = xs[1] - xs[0]

    def h_of(x):
        x = np.asarray(x, dtype=np.float64)
        flat = np.clip(x.reshape(-1), -x0, x0)
        first = np.clip(np.floor((flat + x0) / step).astype(np.int64) - order // 2 + 1, 0, n_table - order)
        out = np.zeros_like(flat)
        for a in range(order):
            xa = xs[first + a]
            basis = np.ones_like(flat)
            for b in range(order):
                if b != a:
                    basis *= (flat - xs[first + b]) / (xa - xs[first + b])
            out += hs[first + a] * basis
        return out.reshape(x.shape)

    return h_of


def misfit_L(weights_fn, h_fn, W, x, nu):
    """L(x, nu) of Eq. csum2 on the outer grid x (nx,) by nu (nn,)."""
    s = tap_offsets(W)
    c = weights_fn(nu)                                      # (nn, W)
    ph = 2.0 * np.pi * (s[None, None, :] - nu[None, :, None]) * x[:, None, None]
    a = (c[None, :, :] * np.exp(1j * ph)).sum(-1)
    return 1.0 - h_fn(x)[:, None] * a


def map_error(weights_fn, h_fn, W, x, n_nu=200):
    """l(x) = int_{-1/2}^{1/2} |L(x, nu)|^2 dnu (Section 3.3)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nq, wn = gauss_legendre(n_nu, -0.5, 0.5)
    L = misfit_L(weights_fn, h_fn, W, x, nq)
    return (wn[None, :] * np.abs(L) ** 2).sum(1)


def error_bound(weights_fn, h_fn, W, x0, nx=200, n_nu=200):
    """E of Eq. norm_bound by tensor Gauss-Legendre quadrature."""
    xq, wx = gauss_legendre(nx, -x0, x0)
    ell = map_error(weights_fn, h_fn, W, xq, n_nu)
    return float(np.sqrt((wx * ell).sum() / (2.0 * x0)))


# -- top hat (Section 6: the original W-stacking seen as W_z = 1) -----------

def tophat_weights(nu):
    """C_z = 1 on |w'| < 1/2, so the single tap weight is 1 for every nu."""
    nu = np.asarray(nu, dtype=np.float64)
    return np.ones(nu.shape + (1,))


def tophat_h(z):
    """h(z) = 1 / sinc z with sinc z = sin(pi z)/(pi z)."""
    return 1.0 / np.sinc(np.asarray(z, dtype=np.float64))


# -- the fit ------------------------------------------------------------------

def _parameter_map(W: int, D: int, nu: np.ndarray):
    """Basis of the even parameterisation: B[p] is (nn, W), c = sum_p beta_p B[p]."""
    s = tap_offsets(W)
    P = _leg.legvander(2.0 * nu, D)                         # (nn, D+1)
    cols = []
    for i, si in enumerate(s):
        if si < 0:
            continue
        for k in range(D + 1):
            if si == 0 and k % 2:
                continue                                    # c_0(nu) is even in nu
            cols.append((i, k))
    B = np.zeros((len(cols), nu.size, W))
    for p, (i, k) in enumerate(cols):
        B[p, :, i] += P[:, k]
        j = W - 1 - i
        if j != i:
            # c_{-s}(nu) = c_s(-nu) and P_k(-2nu) = (-1)^k P_k(2nu)
            B[p, :, j] += (-1.0) ** k * P[:, k]
    return cols, B


def _expand(cols, vec, W, D):
    beta = np.zeros((W, D + 1))
    for (i, k), b in zip(cols, vec):
        beta[i, k] += b
        j = W - 1 - i
        if j != i:
            beta[j, k] += (-1.0) ** k * b
    return beta


def _minimise(W: int, x0: float, degree: int, nx: int, n_nu: int, max_iter: int, vec0=None):
    """Minimise the quadrature form of E^2 over the even-C coefficients, h eliminated.

    Each iteration takes the Gauss-Newton step (least squares on the Jacobian of
    the residual, not the normal equations), halved until E^2 falls.  Where no
    halving helps, it takes a Levenberg-Marquardt step instead: the same least
    squares with the damping term mu |diag(|J_p|) step|^2, mu raised until E^2
    falls.  Stops when neither lowers E^2 or the relative gain is below 1e-10.
    Returns (coefficient vector, parameter map, h at the x nodes, x nodes).
    """
    xq, wx = gauss_legendre(nx, -x0, x0)
    nq, wn = gauss_legendre(n_nu, -0.5, 0.5)
    s = tap_offsets(W)
    cols, B = _parameter_map(W, degree, nq)
    E = np.exp(2j * np.pi * (s[None, None, :] - nq[None, :, None]) * xq[:, None, None])
    A = np.einsum("pnw,xnw->pxn", B, E)                     # d a(x,nu) / d beta_p
    sq = np.sqrt(wx[:, None] * wn[None, :])

    def realify(Z):                                         # complex (p, x, n) -> real rows
        Zw = sq[None] * Z
        return np.concatenate([Zw.real.reshape(Z.shape[0], -1),
                               Zw.imag.reshape(Z.shape[0], -1)], 1).T

    def state(vec):
        a = np.einsum("p,pxn->xn", vec, A)
        R = (wn[None, :] * a.real).sum(1)
        Q = (wn[None, :] * (a.real ** 2 + a.imag ** 2)).sum(1)
        h = R / Q
        rho = 1.0 - h[:, None] * a
        obj = float((wx[:, None] * wn[None, :] * np.abs(rho) ** 2).sum() / (2.0 * x0))
        return a, R, Q, h, rho, obj

    if vec0 is None:
        # start: the best C for h = 1 (one exact partial minimisation)
        y = np.concatenate([sq.ravel(), np.zeros(sq.size)])
        vec = np.linalg.lstsq(realify(A), y, rcond=None)[0]
    else:
        vec = np.asarray(vec0, dtype=np.float64)
    a, R, Q, h, rho, obj = state(vec)
    for _ in range(max_iter):
        dR = (wn[None, None, :] * A.real).sum(2)                                  # (p, x)
        dQ = 2.0 * (wn[None, None, :] * (np.conj(a)[None] * A).real).sum(2)
        dh = dR / Q[None] - (R / Q ** 2)[None] * dQ
        J = realify(-(dh[:, :, None] * a[None] + h[None, :, None] * A))
        rr = np.concatenate([(sq * rho).real.ravel(), (sq * rho).imag.ravel()])
        # one SVD of the column-scaled Jacobian J diag(1/scale) = U S V^T serves both
        # steps: Gauss-Newton (pseudo-inverse, singular values below 1e-14 S_max
        # dropped) and Levenberg-Marquardt (S / (S^2 + mu))
        scale = np.linalg.norm(J, axis=0)
        scale[scale == 0.0] = 1.0
        U, S, Vt = np.linalg.svd(J / scale[None, :], full_matrices=False)
        g = U.T @ rr

        def step_for(filt):
            return -(Vt.T @ (filt * g)) / scale

        keep = S > 1e-14 * S[0]
        step = step_for(np.where(keep, 1.0 / np.where(keep, S, 1.0), 0.0))
        lam, cand = 1.0, None
        while lam > 1e-4:
            trial = state(vec + lam * step)
            if trial[-1] < obj:
                cand, step = trial, lam * step
                break
            lam *= 0.5
        mu = 1e-8
        while cand is None and mu < 1e12:
            step = step_for(S / (S * S + mu))
            trial = state(vec + step)
            if trial[-1] < obj:
                cand = trial
            mu *= 4.0
        if cand is None:
            break
        rel = (obj - cand[-1]) / obj
        vec = vec + step
        a, R, Q, h, rho, obj = cand
        if rel < 1e-10:
            break
    return vec, cols, h, xq


# Above this cropping parameter the fit is followed from x0 = 1/4 upward.
_CONTINUE_ABOVE = 0.3
_CONTINUE_STEP = 0.05


@lru_cache(maxsize=64)
def least_misfit(W: int, x0: float, degree: int = 20, nx: int = 64,
                 n_nu: int = 64, max_iter: int = 60) -> LeastMisfit:
    """Minimise E over even C (support W) and real h for cropping parameter x0.

    For x0 above 0.3 the minimiser is followed from x0 = 1/4 in steps of 0.05,
    each fit starting from the previous one's coefficients: started cold at
    large x0 (from the best C for h = 1), the iteration can settle in a poorer
    local minimum, which it did at W = 8, 12 and 14 with x0 = 0.4 - 0.45 (E
    then fails to fall with W).
    """
    if not (1 <= W <= 16) or not (0.0 < x0 <= 0.5):
        raise ValueError("need 1 <= W <= 16 and 0 < x0 <= 0.5")
    path = [float(x0)]
    if x0 > _CONTINUE_ABOVE:
        path = [0.25]
        while path[-1] + _CONTINUE_STEP < x0 - 1e-12:
            path.append(path[-1] + _CONTINUE_STEP)
        path.append(float(x0))
    vec = None
    for xs in path:
        vec, cols, h, xq = _minimise(W, xs, degree, nx, n_nu, max_iter, vec)
    beta = _expand(cols, vec, W, degree)
    beta = beta * h[np.argmin(np.abs(xq))]                  # gauge: h(0) ~ 1 (h scales as 1/beta)
    lm = LeastMisfit(W=W, x0=float(x0), beta=beta, E=float("nan"))
    Efine = error_bound(lm.weights, lm.h, W, x0)
    return LeastMisfit(W=W, x0=float(x0), beta=beta, E=Efine)
