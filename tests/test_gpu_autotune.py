"""Launch-shape autotuner (psso_autotune): the tuned shape is one of the
candidates it timed, a repeated call is answered from the cache, and a handle
made with the tuned configuration computes exactly what the default handle
and the oracle compute (the launch shape never changes results)."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def _oracle(p, t):
    return oracle.run_problem(p, t)


def _states(lib, ps, t, precision, **cfg):
    h = lib.psso_create_ex(ps, precision, log_stride=1, log_capacity=t + 1, **cfg)
    try:
        lib.psso_run(h, t)
        out = []
        for k, p in enumerate(ps):
            X, P, pF = lib.psso_get_state(h, k, p["N"], p["D"])
            out.append(dict(X=X, P=P, pF=pF, log=lib.psso_get_log(h, k),
                            best=lib.psso_best(h, k, p["D"])))
        return out, lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)


def test_single_swarm_persistent_kernel(lib):
    """Shifted Rastrigin D=100, N=1024 (one swarm over many pipelined blocks):
    particles per block are tuned; results equal the default shape's and the
    oracle's decisions."""
    p = workload.problem("rastrigin", 1024, 100, seed=1, lattice="f32", shift_range=(-4.0, 4.0))
    fields, rep = lib.psso_autotune([p], "f32", generations=100)
    assert rep["candidates"] >= 2
    assert 0 < rep["best_ms"] <= rep["default_ms"]
    assert rep["threads_per_block"] == fields["threads_per_block"]
    assert fields["threads_per_block"] == 0 or fields["threads_per_block"] % 32 == 0
    # cached: nothing is timed again, same answer
    fields2, rep2 = lib.psso_autotune([p], "f32", generations=100)
    assert rep2["candidates"] == 0 and fields2 == fields and rep2["best_ms"] == rep["best_ms"]

    t = 25
    tuned, st = _states(lib, [p], t, "f32", **fields)
    base, _ = _states(lib, [p], t, "f32")
    r = _oracle(p, t)
    for a in (tuned[0], base[0]):
        assert np.array_equal(a["X"], r["X"]) and np.array_equal(a["P"], r["P"])
        assert np.array_equal(a["log"]["index"], r["log_b"])
        assert np.array_equal(a["log"]["accepted"], r["log_acc"])
    assert tuned[0]["best"][0] == base[0]["best"][0] == r["log_v"][t]
    if fields["threads_per_block"]:
        assert st["threads_per_block"] == fields["threads_per_block"]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batched_pipeline(lib, precision):
    """24 swarms of mixed width on the batched pipeline: blocks per SM of the
    step kernels are tuned; every instance is unchanged by the tuned shape."""
    fns = ["sphere", "rastrigin", "rosenbrock", "ackley"]
    rng = np.random.default_rng(11)
    ps = [workload.problem(fns[k % 4], int(rng.integers(40, 400)),
                           int([5, 30, 100, 150, 300, 700][k % 6]), seed=7, lattice="f32",
                           stream=k) for k in range(24)]
    fields, rep = lib.psso_autotune(ps, precision, generations=20)
    assert rep["candidates"] >= 2
    assert 0 < rep["best_ms"] <= rep["default_ms"]
    assert fields["threads_per_block"] == 0
    assert 0 <= fields["batch_blocks_per_sm"] <= 8
    t = 8
    tuned, st = _states(lib, ps, t, precision, **fields)
    base, _ = _states(lib, ps, t, precision)
    assert st["batch_classes"] > 0 and st["blocks"] == 0
    for a, b in zip(tuned, base):
        assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["P"], b["P"])
        assert np.array_equal(a["log"]["index"], b["log"]["index"])
        assert a["best"][0] == b["best"][0]
    for k in (0, 5, 17):
        r = _oracle(ps[k], t)
        assert np.array_equal(tuned[k]["X"], r["X"]) and np.array_equal(tuned[k]["P"], r["P"])


def test_tensor_pipeline_has_fixed_shape(lib):
    """A rotated swarm on the tensor-core pipeline adds no candidates."""
    p = workload.problem("rot_rastrigin", 256, 64, seed=3, lattice="f32")
    fields, rep = lib.psso_autotune([p], "f32", generations=5)
    assert rep["candidates"] == 1
    assert fields == {"threads_per_block": 0, "batch_blocks_per_sm": 0}
    assert rep["best_ms"] == rep["default_ms"] > 0


def test_rejects_bad_arguments(lib):
    p = workload.problem("sphere", 64, 10, seed=1)
    with pytest.raises(lib.PssoError):
        lib.psso_autotune([p], "f64", generations=0)
    with pytest.raises(lib.PssoError):
        lib.psso_create_ex([p], "f64", batch_blocks_per_sm=-1)
