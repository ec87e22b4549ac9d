"""The multi-GPU path of bench.py is replicas only: each rank runs its own copy
of the workload, the ranks meet at a barrier, and the job's time is the slowest
rank's.  Checked with two gloo processes on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
        slowest = bench.max_over_ranks(ms)
        dist.barrier()
        with open(os.path.join(out, f"rank{rank}.txt"), "w") as f:
            f.write(f"{slowest!r} {bench.replica_value(1000, world, slowest)!r}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [tuple(float(x) for x in (tmp_path / f"rank{r}.txt").read_text().split()) for r in range(2)]
    assert res[0] == res[1] == (15.0, 1000 * 2 / 0.015)


def test_single_process_is_a_no_op():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(10, 1, 1000.0) == 10.0
