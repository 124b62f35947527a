"""The bench's multi-rank path on CPU: two gloo ranks (replicas, weak scaling).

Each rank times its own replica; the job time is the slowest rank's (all-reduce MAX after a
barrier), and the whole-job throughput is world x units per rank / that time.  The reference
arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = [40.0, 55.0][rank]                      # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world)
        out[rank] = (ms_max, bench.job_throughput(1000, world, ms_max))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        got = dict(out)
    assert got[0][0] == got[1][0] == 55.0
    assert got[0][1] == pytest.approx(2 * 1000 / 0.055)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse.__globals__["argparse"].Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None
