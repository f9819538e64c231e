"""The paper's own timing workload (Rosenbrock, D=50, Table 3.10) with its
Cw/Cp/Cg = 0.3/0.6/0.8 triple in the interval order Eq. 2.1 prints (keep,
pBest, gBest, fresh): the GPU run is bit-identical to the oracle, with the
FP64 fitness and in the FP32-with-recheck form (identical decisions); the
empirical branch frequencies match the paper's interval widths; the same
branch probabilities in the default order (gBest, pBest, keep) give another,
equally exact trajectory."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def _gpu(lib, p, t, precision):
    h = lib.psso_create_ex([p], precision, log_stride=1, log_capacity=t + 1)
    try:
        lib.psso_run(h, t)
        X, P, pF = lib.psso_get_state(h, 0, p["N"], p["D"])
        log = lib.psso_get_log(h, 0)
    finally:
        lib.psso_destroy(h)
    return X, P, pF, log


@pytest.mark.parametrize("N", [100, 350])
def test_paper_rosenbrock_bitexact(lib, N):
    cfg = workload.config(f"paper_rosenbrock_n{N}")
    p = cfg["problems"][0]
    assert p["order"] == "paper"
    t = 40
    X, P, pF, log = _gpu(lib, p, t, "f64")
    r = oracle.run_problem(p, t)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"]) and np.array_equal(pF, r["pF"])
    assert np.array_equal(log["index"], r["log_b"]) and np.array_equal(log["value"], r["log_v"])
    # branch frequencies of the oracle's draws (gBest, pBest, keep, fresh):
    # [Cp, Cg) = 0.2, [Cw, Cp) = 0.3, [0, Cw) = 0.3, [Cg, 1) = 0.2
    n = r["branch"].sum()
    want = np.array([0.2, 0.3, 0.3, 0.2])
    assert np.all(np.abs(r["branch"] / n - want) <= 5 * np.sqrt(want * (1 - want) / n))


def test_paper_order_differs_from_default_order(lib):
    """The same branch probabilities in the default order: another trajectory,
    also bit-identical to the oracle's."""
    p = workload.config("paper_rosenbrock_n100")["problems"][0]
    q = dict(p, order="gpx", Cg=0.2, Cp=0.5, Cw=0.8)
    t = 30
    Xp, _, _, _ = _gpu(lib, p, t, "f64")
    Xq, Pq, pFq, logq = _gpu(lib, q, t, "f64")
    r = oracle.run_problem(q, t)
    assert np.array_equal(Xq, r["X"]) and np.array_equal(Pq, r["P"]) and np.array_equal(pFq, r["pF"])
    assert not np.array_equal(Xp, Xq)


@pytest.mark.parametrize("fn", ["rastrigin", "rot_ackley"])
def test_paper_order_f32_same_decisions(lib, fn):
    p = workload.problem(fn, 200, 50, seed=9, lattice="f32", Cg=0.8, Cp=0.6, Cw=0.3, order="paper")
    t = 30
    X, P, _, log = _gpu(lib, p, t, "f32")
    r = oracle.run_problem(p, t)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    assert np.array_equal(log["index"], r["log_b"])


def test_paper_rosenbrock_f32_lattice_same_decisions(lib):
    cfg = workload.config("paper_rosenbrock_n200")
    p = dict(cfg["problems"][0], lattice="f32")
    t = 40
    X, P, _, log = _gpu(lib, p, t, "f32")
    r = oracle.run_problem(p, t)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    assert np.array_equal(log["index"], r["log_b"])


def test_paper_order_batched_and_tensor_paths(lib):
    """The batched pipeline (16 swarms) and the tensor-core pipeline take the
    paper's order too."""
    ps = [workload.problem("sphere", 70 + k, 20 + 3 * k, seed=2, lattice="f32", stream=k,
                           Cg=0.8, Cp=0.6, Cw=0.3, order="paper") for k in range(16)]
    t = 8
    h = lib.psso_create_ex(ps, "f32", batch_stream=1)
    try:
        lib.psso_run(h, t)
        for k, p in enumerate(ps):
            X, P, _ = lib.psso_get_state(h, k, p["N"], p["D"])
            r = oracle.run_problem(p, t)
            assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    finally:
        lib.psso_destroy(h)
    p = workload.problem("rot_rastrigin", 256, 64, seed=3, lattice="f32", Cg=0.8, Cp=0.6, Cw=0.3,
                         order="paper")
    h = lib.psso_create_ex([p], "f32", tensor_rotation=1)
    try:
        lib.psso_run(h, t)
        X, P, _ = lib.psso_get_state(h, 0, p["N"], p["D"])
        st = lib.psso_stats(h)
    finally:
        lib.psso_destroy(h)
    assert st["blocks"] == 0
    r = oracle.run_problem(p, t)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
