"""The multi-rank host logic of bench.py on CPU (gloo, two ranks): the path
shards by image with no exchange, so ranks render disjoint pose sequences and
the job's time is the slowest rank's (all_reduce MAX)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [bench.replica_pose_index(rank, i) for i in range(40)]
        got = [None] * world
        dist.all_gather_object(got, mine)
        ms = 1.5 + rank   # rank 1 is the slower replica
        dist.barrier()
        worst = bench.max_over_ranks(ms, dist, device="cpu")
        out.put((rank, got, worst))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_poses_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, worst in res:
        assert worst == 2.5                      # the slower rank's time, on every rank
        a, b = set(got[0]), set(got[1])
        assert len(a) == len(b) == 40 and not (a & b)


def test_single_process_keeps_its_value():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_pose_index(0, 7) == 7
