"""bench.py's multi-process oracle harness: splitting the visibilities into slabs by
first-tap plane over spawned processes gives exactly the single-process oracle's
Algorithms 5 and 6 (both are linear in the visibility set)."""
import numpy as np

from gpu_helpers import case, oracle_pair, rel


def test_slab_split_equals_the_single_process_oracle():
    import bench
    from paper_2101_11172_gb300 import synth
    c = case(N=32, M=600, wfac=30.0, seed=5)
    wl = synth.Workload("pool-test", c["N"], c["x0"], c["W"], c["fov"], c["uvw"], c["image"], c["vis"])
    pool = bench.OraclePool(wl, procs=3)
    try:
        parts = pool.slabs(pool.order, int(pool.t0.min()), int(pool.t0.max()))
        assert len(parts) == 3 and sum(p.size for p in parts) == c["M"]
        assert all(np.all(np.diff(pool.t0[p]) >= 0) for p in parts)
        dt, v, d = pool.full_pass()
        assert dt > 0
        step = pool.slab_step(np.random.default_rng(1), 50)
        assert step[1] > 0
    finally:
        pool.close()
    _, _, v_ref, d_ref = oracle_pair(c)
    assert rel(v, v_ref) < 1e-12 and rel(d, d_ref) < 1e-12
