"""The rest of Table 3.2 on the GPU -- f2 hyper-ellipsoid, f3 Schwefel's
problem 1.2, f7 Griewank, f8 Powell, f9 Schwefel -- against the oracle:
whole runs bit-identical with FP64 fitness (persistent kernel, batched
pipeline, asynchronous flow), batched fitness bit-identical, the
hyper-ellipsoid also in the FP32 + recheck form (identical decisions, 1e-6
relative), and the FP32 form refused for the FP64-only functions."""
import numpy as np
import pytest

import oracle
import workload
from helpers import REL_TOL, fitness_rel_err

pytestmark = pytest.mark.gpu

NEW = ["hyper_ellipsoid", "schwefel12", "griewank", "powell", "schwefel"]
FP64_ONLY = ["schwefel12", "griewank", "powell", "schwefel"]


def _run(lib, problems, t, precision="f64", **cfg):
    h = lib.psso_create_ex(problems, precision, log_stride=1, log_capacity=t + 1, **cfg)
    try:
        lib.psso_run(h, t)
        out = []
        for k, p in enumerate(problems):
            X, P, pF = lib.psso_get_state(h, k, p["N"], p["D"])
            out.append(dict(X=X, P=P, pF=pF, log=lib.psso_get_log(h, k),
                            best=lib.psso_best(h, k, p["D"])))
        return out, lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)


def _bitexact(g, r, t):
    assert np.array_equal(g["X"], r["X"])
    assert np.array_equal(g["P"], r["P"])
    assert np.array_equal(g["pF"], r["pF"])
    assert np.array_equal(g["log"]["index"], r["log_b"])
    assert np.array_equal(g["log"]["value"], r["log_v"])
    assert np.array_equal(g["log"]["accepted"], r["log_acc"])
    v, b, row = g["best"]
    assert b == r["log_b"][t] and v == r["log_v"][t] and np.array_equal(row, r["G"])


@pytest.mark.parametrize("fn", NEW)
@pytest.mark.parametrize("lattice", ["f64", "f32"])
@pytest.mark.parametrize("N,D,t", [(37, 5, 20), (130, 129, 6), (9, 257, 4), (33, 31, 15),
                                   (5, 1000, 2), (64, 1, 10)])
def test_fp64_bitexact(lib, fn, lattice, N, D, t):
    p = workload.problem(fn, N, D, seed=7 + N, lattice=lattice, stream=D % 3)
    (g,), _ = _run(lib, [p], t)
    _bitexact(g, oracle.run_problem(p, t), t)


@pytest.mark.parametrize("fn", NEW)
def test_fp64_multiblock_and_async(lib, fn):
    """A swarm over many blocks (record exchange), and the asynchronous flow."""
    p = workload.problem(fn, 1500, 40, seed=5, lattice="f64")
    t = 10
    (g,), st = _run(lib, [p], t, single_block_max=-1)
    assert st["blocks"] > 1
    _bitexact(g, oracle.run_problem(p, t), t)
    (a,), _ = _run(lib, [p], t, flow="async")
    _bitexact(a, oracle.run_problem(p, t, flow="async"), t)


def test_batched_pipeline_mixed(lib):
    ps = [workload.problem(NEW[k % 5], 50 + 7 * k, 10 + 23 * k, seed=3, lattice="f32", stream=k)
          for k in range(20)]
    t = 5
    outs, st = _run(lib, ps, t, batch_stream=1)
    assert st["batch_classes"] >= 1
    for g, p in zip(outs, ps):
        _bitexact(g, oracle.run_problem(p, t), t)


def test_evaluate_fp64_matches_oracle(lib):
    rng = np.random.default_rng(11)
    for fn in NEW:
        lb, ub = workload.BOUNDS[fn]
        for D in (1, 3, 7, 100, 333, 1000):
            X = rng.uniform(lb, ub, (9, D))
            o = workload.shift(D, 0.8 * lb, 0.8 * ub, 2)
            f, _ = lib.psso_evaluate(fn, X, o)
            ref = np.array([oracle.fitness(fn, x, o) for x in X])
            assert np.array_equal(f, ref), (fn, D)


@pytest.mark.parametrize("N,D,t", [(61, 13, 30), (300, 100, 20), (8, 700, 5)])
def test_hyper_ellipsoid_fp32_same_decisions(lib, N, D, t):
    p = workload.problem("hyper_ellipsoid", N, D, seed=21 + D, lattice="f32")
    (g,), _ = _run(lib, [p], t, precision="f32")
    r = oracle.run_problem(p, t)
    assert np.array_equal(g["X"], r["X"]) and np.array_equal(g["P"], r["P"])
    assert np.array_equal(g["log"]["index"], r["log_b"])
    rel = fitness_rel_err(g["pF"], r["pF"], "hyper_ellipsoid")
    assert np.all(rel <= REL_TOL), rel.max()


@pytest.mark.parametrize("fn", FP64_ONLY)
def test_fp32_form_refused(lib, fn):
    p = workload.problem(fn, 20, 8, seed=1, lattice="f32")
    with pytest.raises(lib.PssoError) as e:
        lib.psso_create_ex([p], "f32")
    assert e.value.status == lib.PSSO_ERR_UNSUPPORTED
    X = np.zeros((2, 8))
    with pytest.raises(lib.PssoError) as e:
        lib.psso_evaluate(fn, X, None, precision="f32")
    assert e.value.status == lib.PSSO_ERR_UNSUPPORTED


def test_noalloc_new_functions(lib):
    """The allocation-free batched fitness: the FP64-only functions in FP64, the
    hyper-ellipsoid (weights j + 1 made on the device) in both precisions."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(3)
    for fn, prec in (("griewank", "f64"), ("schwefel12", "f64"), ("powell", "f64"),
                     ("schwefel", "f64"), ("hyper_ellipsoid", "f64"), ("hyper_ellipsoid", "f32")):
        lb, ub = workload.BOUNDS[fn]
        D, N = 77, 40
        o = workload.shift(D, 0.8 * lb, 0.8 * ub, 4, lattice="f32")
        X = rng.uniform(lb, ub, (N, D)).astype(np.float32).astype(np.float64)
        Xd = torch.from_numpy(X).to(dev)
        od = torch.from_numpy(o).to(dev)
        f = torch.empty(N, dtype=torch.float64, device=dev)
        e = torch.empty(N, dtype=torch.float64, device=dev)
        lib.psso_evaluate_noalloc(fn, N, D, Xd.data_ptr(), od.data_ptr(), None, prec, f.data_ptr(),
                                  e.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize()
        ref, ref_e = lib.psso_evaluate(fn, X, o, precision=prec)
        assert np.array_equal(f.cpu().numpy(), ref), fn
        if prec == "f32":
            assert np.array_equal(e.cpu().numpy(), ref_e), fn
