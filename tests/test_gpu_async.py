"""The asynchronous flow (Alg. 1) on the GPU against the oracle's Alg. 1,
element by element: positions, pBests, pBest fitness, and the gBest index and
value of every generation bit-identical (FP64 fitness), for every test
function, both lattices, both interval orders, swarms on one block and on
many, split runs, reset and checkpoint / resume."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

FNS = ["sphere", "ellipsoid", "rastrigin", "rosenbrock", "ackley", "rot_ellipsoid",
       "rot_rastrigin", "rot_ackley", "hyper_ellipsoid", "schwefel12", "griewank", "powell",
       "schwefel"]


def _gpu(lib, p, t, chunks=None, **cfg):
    h = lib.psso_create_ex([p], "f64", flow="async", log_stride=1, log_capacity=t + 1, **cfg)
    try:
        for c in (chunks or [t]):
            lib.psso_run(h, c)
        X, P, pF = lib.psso_get_state(h, 0, p["N"], p["D"])
        log = lib.psso_get_log(h, 0)
        best = lib.psso_best(h, 0, p["D"])
        st = lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)
    return dict(X=X, P=P, pF=pF, log=log, best=best), st


def _same(g, r, t):
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


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("N,D,t", [(37, 5, 30), (300, 31, 12), (9, 257, 6), (2000, 16, 5)])
def test_async_bitexact(lib, fn, N, D, t):
    p = workload.problem(fn, N, D, seed=5 + N, lattice="f64", stream=D % 5)
    g, st = _gpu(lib, p, t)
    _same(g, oracle.run_problem(p, t, flow="async"), t)


@pytest.mark.parametrize("order", ["gpx", "paper"])
@pytest.mark.parametrize("lattice", ["f64", "f32"])
def test_async_orders_and_lattices(lib, order, lattice):
    kw = dict(Cg=0.4, Cp=0.7, Cw=0.9) if order == "gpx" else dict(Cg=0.8, Cp=0.6, Cw=0.3)
    p = workload.problem("rastrigin", 700, 40, seed=2, lattice=lattice, order=order, **kw)
    t = 20
    g, st = _gpu(lib, p, t)
    assert st["blocks"] >= 1
    _same(g, oracle.run_problem(p, t, flow="async"), t)


def test_async_differs_from_sync(lib):
    p = workload.problem("sphere", 200, 20, seed=1)
    t = 10
    g, _ = _gpu(lib, p, t)
    r_async = oracle.run_problem(p, t, flow="async")
    r_sync = oracle.run_problem(p, t, flow="sync")
    _same(g, r_async, t)
    assert not np.array_equal(g["X"], r_sync["X"])


def test_async_many_blocks_split_runs_reset_and_resume(lib):
    """A swarm over many blocks (grid barrier between rounds); the generations
    split over several calls, a reset, and a checkpoint resumed in another
    handle give the uninterrupted run."""
    p = workload.problem("ackley", 6000, 24, seed=4)
    t = 12
    r = oracle.run_problem(p, t, flow="async")
    g, st = _gpu(lib, p, t, chunks=[1, 4, 7])
    assert st["blocks"] > 1
    _same(g, r, t)
    h = lib.psso_create_ex([p], "f64", flow="async")
    h2 = lib.psso_create_ex([p], "f64", flow="async")
    try:
        lib.psso_run(h, 3)
        lib.psso_reset(h)
        lib.psso_run(h, 5)
        lib.psso_load(h2, lib.psso_save(h))
        lib.psso_run(h2, t - 5)
        X, P, pF = lib.psso_get_state(h2, 0, p["N"], p["D"])
    finally:
        lib.psso_destroy(h)
        lib.psso_destroy(h2)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"]) and np.array_equal(pF, r["pF"])


def test_async_rejects_what_it_does_not_run(lib):
    p = workload.problem("sphere", 50, 8, seed=1, lattice="f32")
    with pytest.raises(lib.PssoError) as e:
        lib.psso_create_ex([p], "f32", flow="async")
    assert e.value.status == lib.PSSO_ERR_UNSUPPORTED
    with pytest.raises(lib.PssoError) as e:
        lib.psso_create_ex([p, dict(p, sid=1)], "f64", flow="async")
    assert e.value.status == lib.PSSO_ERR_UNSUPPORTED
