"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas
get disjoint image seeds, the step time is the max over ranks, and the job
value counts the units of every rank."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    t = bench.reduce_max_time(1.0 + rank, dist, torch.device("cpu"))
    seeds = bench.rank_seeds(rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (t, gathered, bench.job_value(10.0, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas():
    ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pp = os.environ.get("PYTHONPATH", "")
    if ROOT not in pp.split(os.pathsep):
        os.environ["PYTHONPATH"] = ROOT + (os.pathsep + pp if pp else "")
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    for r in range(2):
        t, gathered, value = out[r]
        assert t == 2.0                             # slowest rank
        assert value == 10.0 * 2 / 2.0
        assert set(gathered[0]).isdisjoint(gathered[1])
