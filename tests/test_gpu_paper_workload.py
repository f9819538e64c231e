"""The paper's own timing workload (Rosenbrock, D=50, Table 3.10) with its
Cw/Cp/Cg = 0.3/0.6/0.8 triple taken by probability (cumulative 0.2/0.5/0.8):
the GPU run is bit-identical to the oracle, with the FP64 fitness and in the
FP32-with-recheck form (identical decisions), and the empirical branch
frequencies match the paper's interval widths."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [100, 350])
def test_paper_rosenbrock_bitexact(lib, N):
    cfg = workload.config(f"paper_rosenbrock_n{N}")
    p = cfg["problems"][0]
    t = 40
    h = lib.psso_create_ex([p], "f64", log_stride=1, log_capacity=t + 1)
    try:
        lib.psso_run(h, t)
        X, P, pF = lib.psso_get_state(h, 0, p["N"], p["D"])
        log = lib.psso_get_log(h, 0)
    finally:
        lib.psso_destroy(h)
    r = oracle.run(p["fn"], p["N"], p["D"], p["lb"], p["ub"], p["Cg"], p["Cp"], p["Cw"],
                   p["seed"], t, o=p["o"])
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"]) and np.array_equal(pF, r["pF"])
    assert np.array_equal(log["index"], r["log_b"]) and np.array_equal(log["value"], r["log_v"])
    # branch frequencies of the oracle's draws: gBest 0.2, pBest 0.3, keep 0.3, fresh 0.2
    n = r["branch"].sum()
    want = np.array([0.2, 0.3, 0.3, 0.2])
    assert np.all(np.abs(r["branch"] / n - want) <= 5 * np.sqrt(want * (1 - want) / n))


def test_paper_rosenbrock_f32_lattice_same_decisions(lib):
    cfg = workload.config("paper_rosenbrock_n200")
    p = dict(cfg["problems"][0], lattice="f32")
    t = 40
    h = lib.psso_create_ex([p], "f32", log_stride=1, log_capacity=t + 1)
    try:
        lib.psso_run(h, t)
        X, P, _ = lib.psso_get_state(h, 0, p["N"], p["D"])
        log = lib.psso_get_log(h, 0)
    finally:
        lib.psso_destroy(h)
    r = oracle.run(p["fn"], p["N"], p["D"], p["lb"], p["ub"], p["Cg"], p["Cp"], p["Cw"],
                   p["seed"], t, lattice="f32", o=p["o"])
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"])
    assert np.array_equal(log["index"], r["log_b"])
