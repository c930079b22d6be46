"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica (the path does not shard: replicas only), combine to the whole-job
value = V-cycles of all ranks x DoFs / the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r did 3 + r V-cycles on 1000 DoFs in 0.5 + r seconds
        value, t_max = bench.whole_job_mdofs(dist, "cpu", 1000, 3 + rank, 0.5 + rank)
        out[rank] = (value, t_max)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_whole_job_value():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    expect = 1000 * (3 + 4) / 1.5 / 1e6
    for r in range(world):
        value, t_max = res[r]
        assert t_max == pytest.approx(1.5)
        assert value == pytest.approx(expect)


def test_one_rank_is_the_plain_value():
    sys.path.insert(0, ROOT)
    import bench
    value, t_max = bench.whole_job_mdofs(None, "cpu", 2000, 7, 0.25)
    assert t_max == 0.25 and value == pytest.approx(2000 * 7 / 0.25 / 1e6)
