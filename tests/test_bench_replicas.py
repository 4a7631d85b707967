"""The replica logic of bench.py under torch.distributed (gloo, two ranks on
the CPU): every rank gets its own instance seed, and the step time reported
is the slowest rank's."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(2, rank))
    out[rank] = (ms, seeds)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_and_solve_different_instances():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert [res[r][0] for r in range(world)] == [15.0, 15.0]
    seeds = res[0][1]
    assert len(set(seeds)) == world and res[1][1] == seeds


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.replica_seed(2, 0) == 2
