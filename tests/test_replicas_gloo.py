"""Host logic of the multi-GPU replicas path (bench.py under torchrun), run as
two gloo ranks on the CPU: each rank's instances draw from Philox streams no
other instance of the job uses, the step time is the maximum over ranks, and
the job's rate counts every rank's units over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import bench
    import workload
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        problems = workload.config("batched_512")["problems"][:6]
        mine = bench.replica_problems(problems, rank)
        sids = [None] * world
        dist.all_gather_object(sids, [p["sid"] for p in mine])
        own_ms = 10.0 + 5.0 * rank              # rank 1 is the slow one
        total = bench.max_over_ranks(own_ms, dist, "cpu")
        rate = bench.job_rate(1000, 4, world, total)
        q.put((rank, sids, total, rate, [p["N"] for p in mine]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    sids = out[0][1]
    flat = [s for r in sids for s in r]
    assert len(set(flat)) == len(flat)                 # no two instances share a stream
    assert sids[0] == list(range(6)) and sids[1] == list(range(6, 12))
    for rank, _, total, rate, Ns in out:
        assert total == 15.0                           # the slowest rank's time
        assert rate == pytest.approx(1000 * 4 * 2 / 0.015)
        assert Ns == out[0][4]                         # same workload on every rank


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    ps = [dict(sid=3, N=1), dict(sid=4, N=2)]
    assert [p["sid"] for p in bench.replica_problems(ps, 0)] == [3, 4]
