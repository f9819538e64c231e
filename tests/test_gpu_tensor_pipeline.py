"""Rotated functions with FP32 fitness + FP64 recheck on the tensor-core
generation pipeline (tensor_rotation=1): every decision equal to the FP64
oracle's, so positions, pBests and the gBest index at every generation are
bit-identical to the oracle; fitness intervals contain the oracle's values."""
import numpy as np
import pytest

import oracle
import workload
from helpers import REL_TOL, fitness_rel_err

pytestmark = pytest.mark.gpu

ROT = ["rot_ellipsoid", "rot_rastrigin", "rot_ackley"]


def _oracle(p, t):
    return oracle.run_problem(p, t)


def _run(lib, problems, t, chunks=None, **cfg):
    cfg.setdefault("tensor_rotation", 1)
    h = lib.psso_create_ex(problems, "f32", log_stride=1, log_capacity=t + 1, **cfg)
    try:
        for c in (chunks or [t]):
            lib.psso_run(h, c)
        out = []
        for k, p in enumerate(problems):
            X, P, pF = lib.psso_get_state(h, k, p["N"], p["D"])
            out.append(dict(X=X, P=P, pF=pF, log=lib.psso_get_log(h, k),
                            best=lib.psso_best(h, k, p["D"])))
        return out, lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)


def _same(g, r, t, fn):
    assert np.array_equal(g["X"], r["X"])
    assert np.array_equal(g["P"], r["P"])
    rel = fitness_rel_err(g["pF"], r["pF"], fn)
    assert np.all(rel <= REL_TOL), rel.max()
    log = g["log"]
    assert np.array_equal(log["generation"], np.arange(t + 1))
    assert np.array_equal(log["index"], r["log_b"])
    assert np.array_equal(log["accepted"], r["log_acc"])
    lo = log["value_lo"].astype(np.float64)
    hi = log["value_hi"].astype(np.float64)
    assert np.all(lo <= r["log_v"]) and np.all(r["log_v"] <= hi)
    v, b, row = g["best"]
    assert b == r["log_b"][t] and v == r["log_v"][t]
    assert np.array_equal(row, r["G"])


@pytest.mark.parametrize("fn", ROT)
@pytest.mark.parametrize("N,D,t", [(128, 32, 30), (300, 100, 25), (1000, 64, 15), (257, 1000, 4),
                                   (130, 1, 10), (1, 40, 12), (200, 129, 20)])
def test_same_decisions_as_oracle(lib, fn, N, D, t):
    p = workload.problem(fn, N, D, seed=40 + D, lattice="f32", stream=N % 3)
    (g,), st = _run(lib, [p], t)
    _same(g, _oracle(p, t), t, fn)
    assert st["blocks"] == 0          # no persistent-kernel blocks: the pipeline ran it


def test_split_runs_and_reset(lib):
    p = workload.problem("rot_rastrigin", 333, 70, seed=3, lattice="f32")
    t = 24
    r = _oracle(p, t)
    (g,), _ = _run(lib, [p], t, chunks=[1, 7, 16])
    _same(g, r, t, p["fn"])
    h = lib.psso_create_ex([p], "f32", tensor_rotation=1, log_stride=1, log_capacity=t + 1)
    try:
        lib.psso_run(h, 9)
        lib.psso_reset(h)
        lib.psso_run(h, t)
        X, P, pF = lib.psso_get_state(h, 0, p["N"], p["D"])
        assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    finally:
        lib.psso_destroy(h)


def test_save_load(lib):
    p = workload.problem("rot_ackley", 260, 48, seed=5, lattice="f32")
    t1, t2 = 8, 9
    r = _oracle(p, t1 + t2)
    h = lib.psso_create_ex([p], "f32", tensor_rotation=1)
    h2 = lib.psso_create_ex([p], "f32", tensor_rotation=1)
    try:
        lib.psso_run(h, t1)
        blob = lib.psso_save(h)
        lib.psso_run(h2, 3)
        lib.psso_load(h2, blob)
        lib.psso_run(h2, t2)
        X, P, pF = lib.psso_get_state(h2, 0, p["N"], p["D"])
        assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
        v, b, row = lib.psso_best(h2, 0, p["D"])
        assert b == r["log_b"][-1] and v == r["log_v"][-1]
    finally:
        lib.psso_destroy(h)
        lib.psso_destroy(h2)


def test_mixed_batch(lib):
    """Rotated instances on the pipeline next to plain ones on the persistent
    kernel, in one handle: each equals its own oracle run."""
    ps = [workload.problem("rosenbrock", 200, 40, seed=8, lattice="f32"),
          workload.problem("rot_ackley", 256, 64, seed=9, lattice="f32"),
          workload.problem("rastrigin", 90, 17, seed=10, lattice="f32"),
          workload.problem("rot_ellipsoid", 140, 33, seed=11, lattice="f32")]
    t = 15
    outs, st = _run(lib, ps, t)
    for g, p in zip(outs, ps):
        _same(g, _oracle(p, t), t, p["fn"])
    assert st["blocks"] > 0


def test_same_as_persistent_kernel(lib):
    p = workload.problem("rot_rastrigin", 256, 96, seed=12, lattice="f32")
    t = 20
    (a,), _ = _run(lib, [p], t, tensor_rotation=1)
    (b,), st = _run(lib, [p], t, tensor_rotation=-1)
    assert st["blocks"] > 0
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["P"], b["P"])
    assert np.array_equal(a["log"]["index"], b["log"]["index"])


def test_polish_on_pipeline_instance(lib):
    p = workload.problem("rot_ackley", 300, 64, seed=13, lattice="f32")
    h = lib.psso_create_ex([p], "f32", tensor_rotation=1)
    try:
        lib.psso_run(h, 20)
        v0 = lib.psso_best(h, 0)[0]
        lib.psso_polish(h, 0, 20, 0.1)
        v1, b, row = lib.psso_best(h, 0, p["D"])
        assert v1 <= v0
        assert v1 == oracle.fitness(p["fn"], row, p["o"], p["w"], p["M"])
        lib.psso_run(h, 10)
        v2 = lib.psso_best(h, 0)[0]
        assert v2 <= v1
    finally:
        lib.psso_destroy(h)


def test_time_kernels_keeps_the_trajectory(lib):
    p = workload.problem("rot_ellipsoid", 256, 80, seed=14, lattice="f32")
    t1, t2 = 5, 7
    h = lib.psso_create_ex([p], "f32", tensor_rotation=1)
    try:
        lib.psso_run(h, t1)
        ms = lib.psso_time_kernels(h, 0, t2)
        assert len(ms) == 11 and all(v > 0 for v in ms.values())
        assert lib.psso_generation(h) == t1 + t2
        X, P, pF = lib.psso_get_state(h, 0, p["N"], p["D"])
        st = lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)
    r = _oracle(p, t1 + t2)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    assert st["launches"] == (1 + 11) + (1 + 11 * t1) + (1 + 11 * t2)
    h = lib.psso_create_ex([p], "f32", tensor_rotation=-1)
    try:
        with pytest.raises(lib.PssoError):
            lib.psso_time_kernels(h, 0, 2)
    finally:
        lib.psso_destroy(h)


@pytest.mark.parametrize("fn", ["rot_ellipsoid", "rot_rastrigin"])
def test_largest_exact_extent(lib, fn):
    """D = 1023 is the largest extent at which the slice GEMM's partial sums stay
    below 2^24 with every slice at its bound (64): the pipeline runs it with the
    oracle's decisions.  D = 1024 is refused when the pipeline is forced and runs
    on the per-particle kernel in the automatic mode."""
    t = 3
    p = workload.problem(fn, 130, 1023, seed=9, lattice="f32")
    (g,), st = _run(lib, [p], t)
    _same(g, _oracle(p, t), t, fn)
    assert st["blocks"] == 0
    q = workload.problem(fn, 130, 1024, seed=9, lattice="f32")
    with pytest.raises(lib.PssoError) as exc:
        lib.psso_create_ex([q], "f32", tensor_rotation=1)
    assert exc.value.status == lib.PSSO_ERR_UNSUPPORTED
    (g,), st = _run(lib, [q], 2, tensor_rotation=0)
    assert st["blocks"] > 0
    _same(g, _oracle(q, 2), 2, fn)
