"""GPU parity: the CUDA path against the CPU oracle, element by element.

FP64 fitness: positions, pBests, pBest fitness and the gBest index / value at
every generation bit-identical to the oracle.  FP32 fitness with FP64 recheck:
identical decisions (so identical positions, pBests and gBest indices) and
fitness within its rigorous bound and 1e-6 relative of the oracle's FP64."""
import numpy as np
import pytest

import oracle
import workload
from helpers import REL_TOL, fitness_rel_err

pytestmark = pytest.mark.gpu


def _gpu_run(lib, problems, t, precision="f64", chunks=None, **cfg):
    h = lib.psso_create_ex(problems, precision, log_stride=1, log_capacity=t + 1, **cfg)
    try:
        for c in (chunks or [t]):
            lib.psso_run(h, c)
        out = []
        for k, p in enumerate(problems):
            X, P, pF = lib.psso_get_state(h, k, p["N"], p["D"])
            log = lib.psso_get_log(h, k)
            v, b, row = lib.psso_best(h, k, p["D"])
            out.append(dict(X=X, P=P, pF=pF, log=log, best=(v, b, row)))
        stats = lib.psso_stats(h)
        return out, stats
    finally:
        lib.psso_destroy(h)


def _oracle_run(p, t):
    return oracle.run_problem(p, t)


def _assert_bitexact(g, r, t):
    assert np.array_equal(g["X"], r["X"])
    assert np.array_equal(g["P"], r["P"])
    assert np.array_equal(g["pF"], r["pF"])
    log = g["log"]
    assert np.array_equal(log["generation"], np.arange(t + 1))
    assert np.array_equal(log["index"], r["log_b"])
    assert np.array_equal(log["value"], r["log_v"])
    assert np.array_equal(log["accepted"], r["log_acc"])
    v, b, row = g["best"]
    assert b == r["log_b"][t] and v == r["log_v"][t]
    assert np.array_equal(row, r["G"])


def test_sphere_d30_full_run_bitexact(lib):
    """The shifted-sphere workload (D=30, N=100, t=1000, FP64 lattice) in full."""
    p = workload.config("sphere_d30")["problems"][0]
    t = 1000
    (g,), _ = _gpu_run(lib, [p], t)
    _assert_bitexact(g, _oracle_run(p, t), t)


CASES = [(37, 5, 30), (130, 129, 8), (9, 257, 5), (64, 1, 25), (33, 31, 20), (5, 1000, 2)]
ALL_FNS = ["sphere", "ellipsoid", "rastrigin", "rosenbrock", "ackley", "rot_ellipsoid",
           "rot_rastrigin", "rot_ackley"]


@pytest.mark.parametrize("fn", ALL_FNS)
@pytest.mark.parametrize("lattice", ["f64", "f32"])
@pytest.mark.parametrize("N,D,t", CASES)
def test_fp64_bitexact(lib, fn, lattice, N, D, t):
    p = workload.problem(fn, N, D, seed=11 + N, lattice=lattice, stream=D % 7)
    (g,), _ = _gpu_run(lib, [p], t)
    _assert_bitexact(g, _oracle_run(p, t), t)


@pytest.mark.parametrize("cfg", [dict(), dict(single_block_max=-1), dict(max_blocks=3),
                                 dict(threads_per_block=64, single_block_max=-1),
                                 dict(threads_per_block=512), dict(residency=2),
                                 dict(residency=2, max_blocks=5, threads_per_block=128),
                                 dict(pipeline=2), dict(threads_per_block=96)])
def test_fp64_multiblock_bitexact(lib, cfg):
    """Swarms spread over many blocks (record exchange between blocks), several
    units per block, and other block sizes give the same trajectory."""
    p = workload.problem("rastrigin", 1500, 40, seed=5, lattice="f32")
    t = 25
    (g,), st = _gpu_run(lib, [p], t, **cfg)
    _assert_bitexact(g, _oracle_run(p, t), t)


def test_split_runs_equal_one_run(lib):
    p = workload.problem("ackley", 700, 64, seed=3, lattice="f64")
    t = 20
    (a,), _ = _gpu_run(lib, [p], t, chunks=[7, 1, 12])
    _assert_bitexact(a, _oracle_run(p, t), t)


def test_reset_restarts_identically(lib):
    p = workload.problem("rastrigin", 400, 50, seed=6, lattice="f32")
    h = lib.psso_create_ex([p], "f32", log_stride=1, log_capacity=32)
    try:
        lib.psso_run(h, 9)
        a = lib.psso_get_state(h, 0, p["N"], p["D"])
        lib.psso_reset(h)
        assert lib.psso_generation(h) == 0
        lib.psso_run(h, 4)
        lib.psso_run(h, 5)
        b = lib.psso_get_state(h, 0, p["N"], p["D"])
        log = lib.psso_get_log(h, 0)
    finally:
        lib.psso_destroy(h)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(log["generation"], np.arange(10))


def test_batched_instances_bitexact(lib):
    table = workload.batched_table(6, seed=4, lattice="f32")
    for q in table:
        q["N"] = min(q["N"], 300)
        q["D"] = min(q["D"], 200)
        q["o"] = q["o"][:q["D"]]
    t = 6
    gs, st = _gpu_run(lib, table, t)
    assert st["instances"] == 6
    for g, p in zip(gs, table):
        _assert_bitexact(g, _oracle_run(p, t), t)


def _assert_same_decisions(g, r, t, fn):
    assert np.array_equal(g["X"], r["X"])
    assert np.array_equal(g["P"], r["P"])
    log = g["log"]
    assert np.array_equal(log["index"], r["log_b"])
    assert np.array_equal(log["accepted"], r["log_acc"])
    lo = log["value_lo"].astype(np.float64)
    hi = log["value_hi"].astype(np.float64)
    assert np.all(lo <= r["log_v"]) and np.all(r["log_v"] <= hi)
    rel = fitness_rel_err(g["pF"], r["pF"], fn)
    assert np.all(rel <= REL_TOL), rel.max()
    v, b, row = g["best"]
    assert b == r["log_b"][t] and v == r["log_v"][t]


@pytest.mark.parametrize("fn", ALL_FNS)
@pytest.mark.parametrize("N,D,t", [(61, 13, 40), (300, 100, 30), (8, 700, 6)])
def test_fp32_recheck_same_decisions(lib, fn, N, D, t):
    p = workload.problem(fn, N, D, seed=21 + D, lattice="f32")
    (g,), _ = _gpu_run(lib, [p], t, precision="f32")
    _assert_same_decisions(g, _oracle_run(p, t), t, fn)


@pytest.mark.parametrize("cfg", [dict(), dict(residency=2), dict(max_blocks=7), dict(pipeline=2),
                                 dict(threads_per_block=128)])
def test_fp32_recheck_multiblock(lib, cfg):
    p = workload.config("rastrigin_d100")["problems"][0]
    t = 60
    (g,), st = _gpu_run(lib, [p], t, precision="f32", **cfg)
    _assert_same_decisions(g, _oracle_run(p, t), t, "rastrigin")
    assert st["blocks"] > 1


def test_evaluate_fp64_matches_oracle(lib):
    rng = np.random.default_rng(0)
    for fn in ALL_FNS:
        for D in (1, 7, 100, 333):
            lb, ub = workload.BOUNDS[fn]
            X = rng.uniform(lb, ub, (17, D))
            o = workload.shift(D, 0.8 * lb, 0.8 * ub, 9)
            w = workload.ellipsoid_weights(D)
            M = workload.rotation(D, 4) if fn.startswith("rot_") else None
            f, _ = lib.psso_evaluate(fn, X, o, w, M)
            ref = np.array([oracle.fitness(fn, x, o, w, M) for x in X])
            assert np.array_equal(f, ref), (fn, D)


@pytest.mark.parametrize("fn", ALL_FNS)
def test_evaluate_fp32_error_bound(lib, fn):
    """|f32 - f64| <= err on random rows and on rows built to stress the
    bound (near-integer and near-half-integer z, tiny z, mixed magnitudes)."""
    rng = np.random.default_rng(1)
    lb, ub = workload.BOUNDS[fn]
    worst_rel = 0.0
    for D in (1, 3, 64, 257, 1000):
        o = workload.shift(D, 0.8 * lb, 0.8 * ub, 5, lattice="f32")
        w = workload.ellipsoid_weights(D)
        M = workload.rotation(D, 6) if fn.startswith("rot_") else None
        rows = [rng.uniform(lb, ub, (64, D))]
        k = rng.integers(-3, 4, (64, D)).astype(np.float64)
        rows.append(o + k + rng.normal(0, 1e-3, (64, D)))
        rows.append(o + k + 0.5 + rng.normal(0, 1e-3, (64, D)))
        rows.append(o + rng.normal(0, 1e-4, (64, D)))
        X = np.clip(np.concatenate(rows), lb, ub).astype(np.float32).astype(np.float64)
        f32, err = lib.psso_evaluate(fn, X, o, w, M, precision="f32")
        f64, _ = lib.psso_evaluate(fn, X, o, w, M, precision="f64")
        assert np.all(np.abs(f32 - f64) <= err), (fn, D)
        floor = 1e-6 * (20 + np.e) if fn.endswith("ackley") else 1e-300
        rel = fitness_rel_err(f32, f64, fn)
        worst_rel = max(worst_rel, float(np.max(rel)))
        # the bound is rigorous but should not be vacuous.  Rotated functions:
        # z = M (x - o) is a compensated FP32 dot product whose error is near
        # u |z| plus (2 gamma^2) sum |M_jk||d_k|; near the optimum, where z
        # cancels, that second part still looks loose relative to f, so those
        # are checked on the uniformly random rows.
        sel = slice(None) if M is None else slice(0, 64)
        assert np.all(err[sel] <= 1e-4 * np.maximum(np.abs(f64[sel]), floor) + 1e-30), (fn, D)
    print(f"{fn}: worst |f32 - f64| / |f64| = {worst_rel:.3e}")
    assert worst_rel <= REL_TOL, worst_rel


def test_timeout_is_reported_not_hung(lib):
    """A block that never publishes: its peers' bounded waits run out and the
    run reports PSSO_ERR_TIMEOUT; the context stays usable."""
    p = workload.problem("sphere", 2000, 16, seed=1)
    h = lib.psso_create_ex([p], single_block_max=-1, spin_limit=20000, fault_skip_rank=2)
    try:
        with pytest.raises(lib.PssoError) as e:
            lib.psso_run(h, 3)
            lib.psso_sync(h)
        assert e.value.status == lib.PSSO_ERR_TIMEOUT
        with pytest.raises(lib.PssoError):
            lib.psso_run(h, 1)
    finally:
        lib.psso_destroy(h)
    # the device is still healthy
    q = workload.problem("sphere", 50, 8, seed=2)
    (g,), _ = _gpu_run(lib, [q], 3)
    _assert_bitexact(g, _oracle_run(q, 3), 3)


def test_save_load_resumes_bitexact(lib):
    p = workload.problem("rosenbrock", 900, 48, seed=8, lattice="f32")
    h = lib.psso_create_ex([p], "f32", log_stride=1, log_capacity=64)
    h2 = lib.psso_create_ex([p], "f32", log_stride=1, log_capacity=64)
    try:
        lib.psso_run(h, 10)
        blob = lib.psso_save(h)
        lib.psso_load(h2, blob)
        assert lib.psso_generation(h2) == 10
        lib.psso_run(h, 15)
        lib.psso_run(h2, 15)
        a = lib.psso_get_state(h, 0, p["N"], p["D"])
        b = lib.psso_get_state(h2, 0, p["N"], p["D"])
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    finally:
        lib.psso_destroy(h)
        lib.psso_destroy(h2)
    r = _oracle_run(p, 25)
    assert np.array_equal(a[0], r["X"]) and np.array_equal(a[1], r["P"])


def test_invalid_arguments(lib):
    bad = [dict(N=0), dict(D=0), dict(D=5000), dict(lb=1.0, ub=1.0), dict(Cg=0.8, Cp=0.5),
           dict(Cw=1.5), dict(fn=99)]
    for b in bad:
        p = workload.problem("sphere", 10, 4, seed=1)
        p.update(b)
        if p["D"] != 4:
            p["o"] = None
        with pytest.raises(lib.PssoError) as e:
            lib.psso_create_ex([p])
        assert e.value.status == lib.PSSO_ERR_ARG
    p = workload.problem("sphere", 10, 4, seed=1, lattice="f64")
    with pytest.raises(lib.PssoError):
        lib.psso_create_ex([p], "f32")          # FP32 fitness needs the F32 lattice
