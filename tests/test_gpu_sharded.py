"""One swarm split into shards (psso_create_shard + psso_set_gbest, the
per-generation exchange of paper_2110_01470_gb300.sharded), driven by one
process on one GPU: the union of the shards' runs equals the oracle's run of
the whole swarm -- positions, pBests and pBest fitness bit for bit with FP64
fitness, identical decisions with FP32 + recheck, and the gBest index and
value of every generation."""
import numpy as np
import pytest

import oracle
import workload
from paper_2110_01470_gb300.sharded import ShardedSwarm

pytestmark = pytest.mark.gpu


def _run(p, t, shards, precision):
    sw = ShardedSwarm(p, precision, shards=shards)
    try:
        sw.run(t)
        X, P, pF = sw.state()
        log = np.array([(i, v) for _, i, v in sw.log])
    finally:
        sw.close()
    return X, P, pF, log


@pytest.mark.parametrize("fn,lattice", [("sphere", "f64"), ("rastrigin", "f32"),
                                        ("rosenbrock", "f64"), ("griewank", "f64"),
                                        ("rot_ackley", "f64")])
@pytest.mark.parametrize("shards", [2, 3])
def test_shards_equal_whole_swarm_fp64(lib, fn, lattice, shards):
    p = workload.problem(fn, 301, 37, seed=4, lattice=lattice)
    t = 12
    X, P, pF, log = _run(p, t, shards, "f64")
    r = oracle.run_problem(p, t)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"]) and np.array_equal(pF, r["pF"])
    assert np.array_equal(log[:, 0], r["log_b"]) and np.array_equal(log[:, 1], r["log_v"])


@pytest.mark.parametrize("fn", ["rastrigin", "rot_rastrigin"])
def test_shards_same_decisions_fp32(lib, fn):
    """FP32 + recheck shards (the rotated one on the tensor-core pipeline: 2 x
    256 particles, D = 64): identical decisions, exact gBest values."""
    p = workload.problem(fn, 512, 64, seed=8, lattice="f32", order="paper", Cg=0.8, Cp=0.6, Cw=0.3)
    t = 10
    X, P, _, log = _run(p, t, 2, "f32")
    r = oracle.run_problem(p, t)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    assert np.array_equal(log[:, 0], r["log_b"]) and np.array_equal(log[:, 1], r["log_v"])


def test_set_gbest_rejects_what_it_cannot_place(lib):
    p = workload.problem("sphere", 2000, 16, seed=1)
    h = lib.psso_create_ex([p], single_block_max=-1)        # spread over several blocks
    try:
        with pytest.raises(lib.PssoError) as e:
            lib.psso_set_gbest(h, 0, 1.0, 0, np.zeros(16))
        assert e.value.status == lib.PSSO_ERR_UNSUPPORTED
    finally:
        lib.psso_destroy(h)
    s = lib.psso_create_shard(p, 100, 50)
    try:
        with pytest.raises(lib.PssoError) as e:
            lib.psso_set_gbest(s, 0, 1.0, 0, np.full(16, 1e9))   # outside [lb, ub]
        assert e.value.status == lib.PSSO_ERR_ARG
    finally:
        lib.psso_destroy(s)
    with pytest.raises(lib.PssoError) as e:
        lib.psso_create_shard(p, 1990, 20)                      # past the swarm's end
    assert e.value.status == lib.PSSO_ERR_ARG


def test_polish_refused_where_the_gbest_is_not_local(lib):
    """A shard's gBest may be another shard's particle: psso_polish refuses
    shard handles.  On a single-block handle whose gBest psso_set_gbest gave
    an index outside the instance, it refuses until a generation has run."""
    p = workload.problem("sphere", 200, 8, seed=2)
    s = lib.psso_create_shard(p, 100, 100)
    try:
        lib.psso_run(s, 2)
        with pytest.raises(lib.PssoError) as e:
            lib.psso_polish(s, 0, steps=2, lr=1e-3)
        assert e.value.status == lib.PSSO_ERR_UNSUPPORTED
    finally:
        lib.psso_destroy(s)
    q = workload.problem("sphere", 100, 8, seed=2)
    h = lib.psso_create_ex([q], single_block_max=1 << 20)      # one block
    try:
        lib.psso_run(h, 2)
        lib.psso_set_gbest(h, 0, 0.5, 150, np.zeros(8))      # an index this instance does not hold
        with pytest.raises(lib.PssoError) as e:
            lib.psso_polish(h, 0, steps=2, lr=1e-3)
        assert e.value.status == lib.PSSO_ERR_STATE
        lib.psso_run(h, 1)                                   # the gBest is a local particle again
        lib.psso_polish(h, 0, steps=2, lr=1e-3)
    finally:
        lib.psso_destroy(h)
