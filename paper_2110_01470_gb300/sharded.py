"""One swarm split over several GPUs (or over several shard handles of one
process): particles are dealt out in contiguous ranges, every shard runs the
update, fitness and pBest step of its own particles on its GPU, and once per
generation the shards agree on the swarm's gBest -- the lowest-index arg-min
of all pBest values (Alg. 4) -- by one exchange: every shard contributes its
own best (FP64 value, global index), the minimum by (value, index) wins, and
its owner broadcasts the row.  The union of the shards' runs is then the run
of the whole swarm bit for bit (the draws are keyed by global particle index).

The exchange is host logic over a small communicator interface:
  * ``DistComm``: torch.distributed (gloo or NCCL), one shard per rank;
  * ``LocalComm``: several shards driven by one process (testing, or one GPU).
The per-generation exchange synchronises the host, so this path trades speed
for size: it is the route for swarms larger than one GPU, not a fast path.
"""
from __future__ import annotations

import numpy as np

from . import (psso_best, psso_create_shard, psso_destroy, psso_get_state, psso_run,
               psso_set_gbest)


def shard_range(N, rank, world):
    """Contiguous particle range [first, first + count) of shard `rank`."""
    first = N * rank // world
    return first, N * (rank + 1) // world - first


def pick_best(cands):
    """Position of the winning candidate among (value, global index) pairs:
    the lowest value, ties to the lowest index (Alg. 4's lowest-index arg-min)."""
    best = 0
    for k in range(1, len(cands)):
        v, i = cands[k]
        bv, bi = cands[best]
        if v < bv or (v == bv and i < bi):
            best = k
    return best


class DistComm:
    """Exchange over torch.distributed: every rank contributes (value, index)
    and the winning rank broadcasts its row."""

    def __init__(self, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        backend = dist.get_backend(group)
        self.device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else \
            torch.device("cpu")

    @property
    def rank(self):
        return self.dist.get_rank(self.group)

    @property
    def world(self):
        return self.dist.get_world_size(self.group)

    def exchange(self, value, index, row):
        """Returns the swarm's (value, index, row) from this rank's candidate."""
        torch, dist = self.torch, self.dist
        mine = torch.tensor([value, float(index)], dtype=torch.float64, device=self.device)
        allc = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(allc, mine, group=self.group)
        cands = [(float(c[0]), int(c[1])) for c in allc]
        w = pick_best(cands)
        buf = torch.tensor(np.asarray(row, dtype=np.float64), device=self.device)
        src = dist.get_global_rank(self.group, w) if self.group is not None else w
        dist.broadcast(buf, src=src, group=self.group)
        return cands[w][0], cands[w][1], buf.cpu().numpy()


class LocalComm:
    """Exchange among candidates that one process already holds."""

    @staticmethod
    def exchange_all(cands_rows):
        w = pick_best([(v, i) for v, i, _ in cands_rows])
        return cands_rows[w]


class ShardedSwarm:
    """A swarm of problem["N"] particles split into shards.

    With ``comm`` (a DistComm) this process owns shard ``comm.rank`` of
    ``comm.world``; without it, it owns all ``shards`` shards itself.
    ``precision`` and ``config`` are those of psso_create_ex."""

    def __init__(self, problem, precision="f64", comm=None, shards=1, **config):
        self.problem, self.comm = problem, comm
        self.N, self.D = int(problem["N"]), int(problem["D"])
        world = comm.world if comm is not None else int(shards)
        mine = [comm.rank] if comm is not None else list(range(world))
        self.ranges = [shard_range(self.N, r, world) for r in range(world)]
        self.own = mine
        self.handles = {}
        try:
            for r in mine:
                first, count = self.ranges[r]
                self.handles[r] = psso_create_shard(problem, first, count, precision, **config)
        except Exception:
            self.close()
            raise
        self.generation = 0
        self.log = []             # (generation, global index, value) of the swarm's gBest
        self._exchange()

    def _exchange(self):
        cands = []
        for r in self.own:
            v, i, row = psso_best(self.handles[r], 0, self.D)
            cands.append((v, self.ranges[r][0] + i, row))
        if self.comm is not None:
            v, i, row = self.comm.exchange(*cands[0])
        else:
            v, i, row = LocalComm.exchange_all(cands)
        for r in self.own:
            psso_set_gbest(self.handles[r], 0, v, i, row)
        self.best = (v, i, row)
        self.log.append((self.generation, i, v))

    def run(self, generations):
        """`generations` more generations, one exchange after each."""
        for _ in range(int(generations)):
            for r in self.own:
                psso_run(self.handles[r], 1)
            self.generation += 1
            self._exchange()

    def state(self):
        """X, P, pF of the particles this process owns (global order)."""
        Xs, Ps, pFs = [], [], []
        for r in self.own:
            count = self.ranges[r][1]
            X, P, pF = psso_get_state(self.handles[r], 0, count, self.D)
            Xs.append(X)
            Ps.append(P)
            pFs.append(pF)
        return np.concatenate(Xs), np.concatenate(Ps), np.concatenate(pFs)

    def close(self):
        for h in self.handles.values():
            psso_destroy(h)
        self.handles = {}
