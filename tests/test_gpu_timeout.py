"""The bounded-wait path of ws_grid, exercised without any fault.

inv_rows (N' = 512 .. 4096) waits on an mbarrier for each plane's TMA row
copy.  WS_WAIT_POLLS = 0 makes that first wait give up at once: every row's
CTA then counts the failure, drains its copy in flight with the full wait
limit and returns, and the call reports WS_ERR_TIMEOUT.  Every copy still
lands, so the context stays usable and the next call on the same plan, with
the knob cleared, must succeed with the right answer.
"""
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


def test_row_copy_wait_gives_up_then_plan_recovers(dev, monkeypatch):
    from paper_2101_11172_gb300 import _lib
    from paper_2101_11172_gb300.wstack import Plan
    c = case(N=256, M=3000, W=7, seed=53)        # N' = 512: compile-time plan with TMA row copies
    with Plan(c["N"], c["x0"], c["W"], c["fov"], c["w_min"], c["w_max"], device=dev) as p:
        assert p.Np == 512
        uvw = torch.from_numpy(c["uvw"]).to(dev)
        vis = torch.from_numpy(c["vis"]).to(torch.complex64).to(dev)
        p.stats(reset=True)
        monkeypatch.setenv("WS_WAIT_POLLS", "0")
        with pytest.raises(_lib.WsError) as err:
            p.grid(uvw, vis)
        assert err.value.status == _lib.WS_ERR_TIMEOUT
        assert "gave up" in str(err.value)
        st = p.stats(reset=True)
        assert st["waits_timed_out"] == c["N"]      # one per image row: every CTA gave up on its first plane
        monkeypatch.delenv("WS_WAIT_POLLS")
        d = p.grid(uvw, vis)
        assert p.last_status == _lib.WS_OK
        torch.cuda.synchronize()
        assert p.stats()["waits_timed_out"] == 0
        d = d.cpu().numpy().astype(np.complex128)
    g, lm, _, d_ref = oracle_pair(c)
    tol = tol_for(c["W"], g.x0)
    assert rel(d, d_ref) < tol
    assert_elementwise(d, d_ref, tol, "grid after a timed-out call")
