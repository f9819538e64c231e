"""bench.py's tensor roofline on a stand-in for the library (no GPU): each
rotated instance is timed early and again around generation t/2, the GEMM
rates follow from the timed GEMM launch, and the refinement share of a
generation counts the refinement and FP64 kernels only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KERNELS = ("update", "gemm_fit", "decide", "z32", "fix32", "z64", "fix64", "argmin0", "z64_argmin",
           "fix64_argmin", "argmin1")


class FakeLib:
    """Records the generations run and hands out kernel times."""

    def __init__(self):
        self.gen = 0
        self.calls = []

    def psso_create_ex(self, problems, prec, stream=None):
        self.gen = 0
        return object()

    def psso_run(self, h, t):
        self.gen += t

    def psso_time_kernels(self, h, instance, generations):
        at = self.gen
        self.gen += generations
        self.calls.append(at)
        late = at >= 100
        ms = {k: 0.01 for k in KERNELS}
        ms["gemm_fit"] = 0.2
        ms["z32"] = 0.02 if late else 0.2
        return ms

    def psso_destroy(self, h):
        pass


def test_early_and_late_timing_and_shares():
    lib = FakeLib()
    p = {"fn": "rot_rastrigin", "N": 8192, "D": 1000}
    r = bench.tensor_roofline(lib, [p], "f32", None, "rotated_d1000", 2000, gens=20)
    assert lib.calls == [20, 1000]
    inst = r["per_instance"][0]
    assert inst["late_generation"] == 1000
    refine = ("z32", "fix32", "z64", "fix64", "z64_argmin", "fix64_argmin")
    for key, ms in (("early", inst["kernels_ms"]), ("late", inst["kernels_ms_late"])):
        want = sum(ms[k] for k in refine) / sum(ms.values())
        assert inst["refine_share"][key] == pytest.approx(want)
    assert inst["refine_share"]["late"] < inst["refine_share"]["early"]
    # 2 N D^2 algorithmic flops and ten slice products over the padded extents per 0.2 ms
    assert r["achieved"] == pytest.approx(2 * 8192 * 1000 ** 2 / 0.2e-3 / 1e12)
    assert r["executed_tflops"] == pytest.approx(10 * 2 * 8192 * 1024 * 1024 / 0.2e-3 / 1e12)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"


def test_short_runs_time_late_after_the_early_window():
    lib = FakeLib()
    p = {"fn": "rot_ackley", "N": 4096, "D": 256}
    bench.tensor_roofline(lib, [p], "f32", None, "grad_d256", 40, gens=20)
    assert lib.calls == [20, 60]          # never before the early window has ended


def test_no_rotated_instance_no_tensor_roofline():
    assert bench.tensor_roofline(FakeLib(), [{"fn": "sphere", "N": 100, "D": 30}], "f32", None, "x", 10) is None
    assert bench.tensor_roofline(FakeLib(), [{"fn": "rot_ackley", "N": 4096, "D": 256}], "f64", None, "x", 10) is None
