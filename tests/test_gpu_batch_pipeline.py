"""Many swarms on the batched throughput pipeline (batch_stream=1): each
instance bit-identical to its own oracle run (FP64 fitness) or with
decisions identical to it (FP32 fitness + FP64 recheck), and identical to
the persistent kernel's results."""
import numpy as np
import pytest

import oracle
import workload
from helpers import REL_TOL, fitness_rel_err

pytestmark = pytest.mark.gpu

FNS = ["sphere", "ellipsoid", "rastrigin", "rosenbrock", "ackley"]


def _oracle(p, t):
    return oracle.run_problem(p, t)


def _mixed(lattice, count=20, seed=0):
    rng = np.random.default_rng(seed)
    ps = []
    for k in range(count):
        fn = FNS[k % len(FNS)]
        D = int([1, 3, 10, 33, 100, 129, 257, 600][k % 8])
        N = int(rng.integers(1, 300))
        ps.append(workload.problem(fn, N, D, seed=100 + k, lattice=lattice, stream=k))
    return ps


def _run(lib, ps, t, precision, chunks=None, **cfg):
    h = lib.psso_create_ex(ps, precision, log_stride=1, log_capacity=t + 1, **cfg)
    try:
        for c in (chunks or [t]):
            lib.psso_run(h, c)
        out = []
        for k, p in enumerate(ps):
            X, P, pF = lib.psso_get_state(h, k, p["N"], p["D"])
            out.append(dict(X=X, P=P, pF=pF, log=lib.psso_get_log(h, k),
                            best=lib.psso_best(h, k, p["D"])))
        return out, lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)


@pytest.mark.parametrize("lattice", ["f64", "f32"])
def test_fp64_bitexact(lib, lattice):
    ps = _mixed(lattice, seed=1)
    t = 12
    outs, st = _run(lib, ps, t, "f64", batch_stream=1)
    assert st["blocks"] == 0
    for g, p in zip(outs, ps):
        r = _oracle(p, t)
        assert np.array_equal(g["X"], r["X"]) and np.array_equal(g["P"], r["P"])
        assert np.array_equal(g["pF"], r["pF"])
        assert np.array_equal(g["log"]["index"], r["log_b"])
        assert np.array_equal(g["log"]["value"], r["log_v"])
        assert np.array_equal(g["log"]["accepted"], r["log_acc"])
        assert np.array_equal(g["best"][2], r["G"])


def test_fp32_same_decisions(lib):
    ps = _mixed("f32", seed=2)
    t = 15
    outs, st = _run(lib, ps, t, "f32", batch_stream=1)
    for g, p in zip(outs, ps):
        r = _oracle(p, t)
        assert np.array_equal(g["X"], r["X"]) and np.array_equal(g["P"], r["P"])
        log = g["log"]
        assert np.array_equal(log["index"], r["log_b"])
        assert np.array_equal(log["accepted"], r["log_acc"])
        lo = log["value_lo"].astype(np.float64)
        hi = log["value_hi"].astype(np.float64)
        assert np.all(lo <= r["log_v"]) and np.all(r["log_v"] <= hi)
        v, b, row = g["best"]
        assert b == r["log_b"][t] and v == r["log_v"][t]
        rel = fitness_rel_err(g["pF"], r["pF"], p["fn"])
        assert np.all(rel <= REL_TOL), (p["fn"], rel.max())


def test_same_as_persistent_kernel_split_runs(lib):
    ps = _mixed("f32", count=24, seed=3)
    t = 10
    a, _ = _run(lib, ps, t, "f32", batch_stream=1, chunks=[1, 2, 7])
    b, st = _run(lib, ps, t, "f32", batch_stream=-1)
    assert st["blocks"] > 0
    for x, y in zip(a, b):
        assert np.array_equal(x["X"], y["X"]) and np.array_equal(x["P"], y["P"])
        assert np.array_equal(x["log"]["index"], y["log"]["index"])


def test_batched_table_sample(lib):
    """The first instances of the 512-swarm table (log-uniform N and D)."""
    ps = workload.config("batched_512")["problems"][:40]
    t = 3
    outs, _ = _run(lib, ps, t, "f32")          # auto: >= 16 swarms -> batched pipeline
    for g, p in zip(outs, ps):
        r = _oracle(p, t)
        assert np.array_equal(g["X"], r["X"]) and np.array_equal(g["P"], r["P"])
        assert np.array_equal(g["log"]["index"], r["log_b"])


def test_reset_save_load(lib):
    ps = _mixed("f64", count=17, seed=4)
    t1, t2 = 4, 5
    h = lib.psso_create_ex(ps, "f64", batch_stream=1)
    h2 = lib.psso_create_ex(ps, "f64", batch_stream=1)
    try:
        lib.psso_run(h, 3)
        lib.psso_reset(h)
        lib.psso_run(h, t1)
        blob = lib.psso_save(h)
        lib.psso_load(h2, blob)
        lib.psso_run(h2, t2)
        for k, p in enumerate(ps):
            r = _oracle(p, t1 + t2)
            X, P, pF = lib.psso_get_state(h2, k, p["N"], p["D"])
            assert np.array_equal(X, r["X"]) and np.array_equal(pF, r["pF"])
    finally:
        lib.psso_destroy(h)
        lib.psso_destroy(h2)
