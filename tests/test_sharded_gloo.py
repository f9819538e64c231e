"""Host logic of one swarm split over several GPUs (paper_2110_01470_gb300.
sharded), run on the CPU: the particle ranges cover the swarm, the gBest is the
lowest-index arg-min over the shards' candidates, and the exchange over
torch.distributed (two gloo ranks) hands every rank the same winner and row."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2110_01470_gb300.sharded import LocalComm, pick_best, shard_range


def test_shard_ranges_cover_the_swarm():
    for N in (1, 7, 100, 1024, 8191):
        for world in (1, 2, 3, 8):
            if world > N:
                continue
            ranges = [shard_range(N, r, world) for r in range(world)]
            assert ranges[0][0] == 0
            for (f0, c0), (f1, _) in zip(ranges, ranges[1:]):
                assert f0 + c0 == f1 and c0 >= 1
            assert sum(c for _, c in ranges) == N


def test_pick_best_is_lowest_index_argmin():
    assert pick_best([(3.0, 5), (1.0, 9), (2.0, 0)]) == 1
    assert pick_best([(1.0, 9), (1.0, 4), (1.0, 7)]) == 1          # ties: lowest index
    assert pick_best([(0.0, 2)]) == 0
    rows = [(1.0, 9, "a"), (1.0, 4, "b")]
    assert LocalComm.exchange_all(rows) == (1.0, 4, "b")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    from paper_2110_01470_gb300.sharded import DistComm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = DistComm()
        assert comm.rank == rank and comm.world == world
        out = []
        # distinct values: the lower one wins wherever it is
        cands = [(5.0, 3), (2.0, 700)]
        v, i, row = comm.exchange(cands[rank][0], cands[rank][1], np.full(4, float(rank)))
        out.append((v, i, row.tolist()))
        # equal values: the lower global index wins
        cands = [(1.0, 9), (1.0, 4)]
        v, i, row = comm.exchange(cands[rank][0], cands[rank][1], np.full(4, 10.0 + rank))
        out.append((v, i, row.tolist()))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_exchange_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        first, second = res[rank]
        assert first == (2.0, 700, [1.0] * 4)        # rank 1's candidate and row
        assert second == (1.0, 4, [11.0] * 4)        # the tie goes to index 4 (rank 1)
