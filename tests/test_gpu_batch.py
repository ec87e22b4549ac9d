"""Batches of independent problems (ws_batch_*): each instance's result is that
of the plain single-instance call, at the plain call's accuracy; the batch's
graph replays, recaptures for new buffers and keeps its answers whatever the
branch count."""
import math

import numpy as np
import pytest

from gpu_helpers import REL_TOL, rel, tol_for
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


def small_batch(n=6):
    """Tiny instances of mixed sizes and counts (the oracle runs them in seconds)."""
    out = []
    for i in range(n):
        rng = synth.rng_for(4, 500 + i)
        N = int(rng.choice([64, 128, 256]))
        M = int(math.exp(rng.uniform(math.log(1e3), math.log(2e4))))
        fov = float(rng.uniform(0.2, 0.4))
        R = 0.45 * N / fov
        uvw = synth.disc_uvw(M, R, 0.05 * R * float(rng.uniform(1.0, 16.0)), rng)
        image = synth.point_sky(N, 12, rng) + 0.1 * synth.complex_normal(N * N, rng).reshape(N, N)
        vis = synth.complex_normal(M, rng)
        out.append(synth.Workload(f"small{i}", N, 0.25, 7, fov, uvw, image, vis))
    return out


def to_dev(wls, dev):
    uvw = [torch.from_numpy(w.uvw).to(dev) for w in wls]
    img = [torch.from_numpy(w.image).to(torch.complex64).to(dev) for w in wls]
    vis = [torch.from_numpy(np.ascontiguousarray(w.vis)).to(torch.complex64).to(dev) for w in wls]
    return uvw, img, vis


def instances(wls):
    return [(w.N, w.fov, w.w_range[0], w.w_range[1], w.M) for w in wls]


def single(w, uvw, img, vis, dev):
    from paper_2101_11172_gb300.wstack import Plan
    with Plan(w.N, w.x0, w.W, w.fov, *w.w_range, device=dev) as p:
        v = p.degrid(img, uvw)
        d = p.grid(uvw, vis)
        torch.cuda.synchronize()
        return v.cpu().numpy().astype(np.complex128), d.cpu().numpy().astype(np.complex128)


def as_np(ts):
    return [t.cpu().numpy().astype(np.complex128) for t in ts]


def test_batch_equals_single_calls_and_oracle(dev):
    from paper_2101_11172_gb300.batch import Batch
    wls = small_batch()
    uvw, img, vis = to_dev(wls, dev)
    with Batch(instances(wls), 0.25, 7, device=dev) as b:
        assert b.branches == 0                       # chosen by the first call
        v = b.degrid(img, uvw)
        assert b.last_status == 0 and b.branches in (1, 2, 4)
        d = b.grid(uvw, vis)
        assert b.last_status == 0
        torch.cuda.synchronize()
        v, d = as_np(v), as_np(d)
        for i, w in enumerate(wls):
            assert (b.info[i].N, b.branch_of(i) >= 0) == (w.N, True)
            v1, d1 = single(w, uvw[i], img[i], vis[i], dev)
            # same kernels; only the plane chunking (and so the summation order) may differ
            assert rel(v[i], v1) < 1e-6 and rel(d[i], d1) < 1e-6, (i, rel(v[i], v1), rel(d[i], d1))
            g = make_geometry(w.N, w.x0, w.W, w.fov, *w.w_range)
            lm = least_misfit(w.W, g.x0)
            tol = tol_for(w.W, g.x0)
            assert rel(v[i], wstack.degrid(g, lm, w.image, w.uvw)) < tol
            assert rel(d[i], wstack.grid(g, lm, w.uvw, w.vis)) < tol


def test_batch_replays_recaptures_and_branch_counts_agree(dev):
    from paper_2101_11172_gb300.batch import Batch
    wls = small_batch(5)
    uvw, img, vis = to_dev(wls, dev)
    with Batch(instances(wls), 0.25, 7, branches=2, device=dev) as b:
        assert b.branches == 2
        v1 = as_np(b.degrid(img, uvw))
        out = [torch.full((w.M,), 7.0, dtype=torch.complex64, device=dev) for w in wls]
        v2 = as_np(b.degrid(img, uvw, out=out))    # new output buffers: a new graph
        v3 = as_np(b.degrid(img, uvw, out=out))    # same buffers: the graph replays
        d1 = as_np(b.grid(uvw, vis))
        for a, c, e in zip(v1, v2, v3):
            assert np.array_equal(a, c) and np.array_equal(a, e)
    with Batch(instances(wls), 0.25, 7, branches=1, device=dev) as b1:
        v4 = as_np(b1.degrid(img, uvw))
        d4 = as_np(b1.grid(uvw, vis))
    for a, c in zip(v1, v4):
        assert rel(a, c) < 1e-6
    for a, c in zip(d1, d4):
        assert rel(a, c) < 1e-6


def test_batch_tuning_waits_for_the_callers_stream(dev):
    # The first call of a batch made with branches = 0 times candidate graphs on the
    # batch's own stream.  Those runs must start only after the work already queued on
    # the caller's stream (here: a long kernel, then a read of the output buffers' old
    # contents, then the copies that produce the inputs), and the caller's stream must
    # wait for them before it goes on.
    from paper_2101_11172_gb300.batch import Batch
    wls = small_batch(4)
    uvw, img, vis = to_dev(wls, dev)
    with Batch(instances(wls), 0.25, 7, branches=1, device=dev) as b1:
        want = as_np(b1.degrid(img, uvw))
    with Batch(instances(wls), 0.25, 7, device=dev) as b:
        assert b.branches == 0
        out = [torch.full((w.M,), 7.0, dtype=torch.complex64, device=dev) for w in wls]
        late = [torch.full_like(u, float("nan")) for u in uvw]
        torch.cuda.synchronize()
        torch.cuda._sleep(int(2e9))                 # about a second of work on the caller's stream
        seen = [o.clone() for o in out]             # queued behind it: the outputs' old contents
        for a, u in zip(late, uvw):
            a.copy_(u)                              # the inputs only now become valid
        got = b.degrid(img, late, out=out)
        torch.cuda.synchronize()
        assert b.last_status == 0 and b.branches in (1, 2, 4)
        for s_ in seen:
            assert bool(torch.all(s_ == 7.0)), "a tuning run wrote an output before the caller's stream read it"
        for a, c in zip(as_np(got), want):
            assert rel(a, c) < 1e-6


def test_batch_reports_the_instance_that_dropped(dev):
    from paper_2101_11172_gb300 import _lib
    from paper_2101_11172_gb300.batch import Batch
    wls = small_batch(3)
    uvw, img, vis = to_dev(wls, dev)
    uvw[1][:, 2] *= 5.0           # instance 1's w now runs far past the range its plan was made for
    with Batch(instances(wls), 0.25, 7, branches=1, device=dev) as b:
        out = b.degrid(img, uvw)
        assert b.last_status == _lib.WS_ERR_W_RANGE
        assert "instance 1" in _lib.ws_last_error()
        torch.cuda.synchronize()
        v1 = out[1].cpu().numpy()
        assert (v1 == 0).any() and (v1 != 0).any()            # dropped ones are zero, the rest computed
        assert all((o.cpu().numpy() != 0).all() for i, o in enumerate(out) if i != 1)


def test_serving_batch_64_instances_against_dft(dev):
    """64 instances, images 512^2 / 1024^2 / 2048^2, 10^4 .. 5x10^6 visibilities each."""
    from paper_2101_11172_gb300.batch import Batch
    wls = synth.batched()
    uvw, img, vis = to_dev(wls, dev)
    with Batch(instances(wls), 0.25, 7, device=dev) as b:
        v = b.degrid(img, uvw)
        d = b.grid(uvw, vis)
        torch.cuda.synchronize()
        assert b.last_status == 0
        errs = []
        for i, w in enumerate(wls):
            g = make_geometry(w.N, w.x0, w.W, w.fov, *w.w_range)
            rng = synth.rng_for(4, 900 + i)
            k = rng.choice(w.M, size=min(64, w.M), replace=False)
            rows, cols = np.nonzero(w.image)
            v_ref = dft.dft_degrid(w.uvw[k], dft.pixel_lmn(g, rows, cols), w.image[rows, cols])
            pr, pc = rng.integers(0, w.N, 4), rng.integers(0, w.N, 4)
            d_ref = dft.dft_grid(w.uvw, w.vis, dft.pixel_lmn(g, pr, pc))
            ev = rel(v[i][torch.from_numpy(k).to(dev)].cpu().numpy().astype(np.complex128), v_ref)
            ed = rel(d[i][pr, pc].cpu().numpy().astype(np.complex128), d_ref)
            errs.append((ev, ed))
        errs = np.array(errs)
        print(f"64 instances on {b.branches} branches: max error vs DFT degrid {errs[:, 0].max():.2e}, "
              f"grid {errs[:, 1].max():.2e}")
        assert errs.max() < REL_TOL
