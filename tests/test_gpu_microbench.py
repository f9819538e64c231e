"""psso_microbench: the measured pipe and latency peaks are positive, mutually
consistent and within the physical limits of the part (no rate above one
operation per lane and clock, the SM clock within the range the driver
reports)."""
import pytest

pytestmark = pytest.mark.gpu


def test_microbench_plausible(lib):
    pk = lib.psso_microbench()
    sms = pk["sms"]
    assert sms >= 1
    mhz = pk["sm_clock_mhz"]
    assert 200.0 < mhz < 3500.0
    lane_clock = sms * 128 * mhz * 1e6          # one operation per lane and clock
    for k in ("fp32_fma_per_s", "int_mad_per_s", "int_mulhi_xor_per_s", "fp64_fma_per_s"):
        assert 0.0 < pk[k] <= 1.05 * lane_clock, k
    # a Philox-4x32-10 block is 20 multiplies and 60 other operations
    assert 0.0 < pk["philox_blocks_per_s"] * 60 <= 1.05 * lane_clock
    for k in ("l2_handoff_ns", "grid_barrier_ns", "cluster_barrier_ns"):
        assert 10.0 < pk[k] < 1e5, k
    # a grid barrier needs at least one hand-off through L2
    assert pk["grid_barrier_ns"] >= 0.5 * pk["l2_handoff_ns"]
