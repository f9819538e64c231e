#!/usr/bin/env python
"""Benchmark of the SSO hot path on GB300 (one JSON line on stdout).

A step is one complete SSO run of the workload -- the initial population and
t generations, each generation = Eq. 2.1 update of every variable + fitness
of every particle + pBest update + gBest arg-min -- through the C ABI.

Default workload: shifted Rastrigin, D=100, N=1024, t=5000, bounds
[-5.12, 5.12], o ~ U[-4,4]^D, FP32 lattice, FP32 fitness with FP64 recheck;
the FP64-fitness path on the same workload is timed beside it.

  value   particle-variable updates / s (N*D*t per step), device-timed with
          CUDA events on the library's stream, state resident in HBM; L2 is
          flushed (256 MiB write) between steps, outside the timed steps
  e2e     the same metric through the public API with host buffers: create
          (problem data host->device), run, best (result device->host),
          destroy, wall-clock with a device sync on both sides
  roofline  the dominant kernel against a measured peak: the persistent
          generation kernel against the pipe rates psso_microbench measures
          in the same run (Philox blocks, FP32 / FP64 FMA, issue); the
          tensor-core GEMM against sustained BF16; the batched step kernel
          against HBM bandwidth
  fitness_err_vs_fp64  FP32 fitness against FP64 on the final state (stored
          pBest values and a raw FP32 evaluation of the same rows)
  peaks   the psso_microbench record of this GPU
  cpu_baseline  the CPU oracle on the host cores, bounded sample

Multi-GPU: replicas only (one independent swarm per rank, stream id = rank,
no collective on the data path); value = all ranks' updates / max time.
`--impl reference` times the CPU oracle on the host cores (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-variable updates/s"
UNIT = "updates/s"
LANES_PER_SM = 128            # 4 sub-partitions x 32 lanes, one warp instruction each per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rastrigin_d100")
    ap.add_argument("--generations", type=int, default=0, help="override t (0 = the workload's)")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--threads-per-block", type=int, default=0,
                    help="fixed block size (0 = the autotuner's choice)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1 = launch shape from psso_autotune (outside the timed steps)")
    ap.add_argument("--polish-steps", type=int, default=2,
                    help="timed runs with the gBest polish (workloads that define one)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def philox_blocks_per_update(p):
    """Philox-4x32-10 blocks one update needs: one rho block per 4 variables,
    plus the fresh-value block(s) of a 4-variable chunk when any of its 4 draws
    selects a fresh value (probability 1 - Cw^4)."""
    fresh_blocks = 1 if p["lattice"] == "f32" else 2
    return 0.25 + fresh_blocks * (1.0 - p["Cw"] ** 4) / 4.0


# Operations of one fitness term: FP32 path (value and error bound) and FP64
# path (sub, the term's arithmetic, the accumulation; sin(pi z) is a degree-21
# odd polynomial after the reduction).
FIT32_OPS = {"sphere": 3, "ellipsoid": 4, "rastrigin": 17, "rosenbrock": 9, "ackley": 19}
FIT64_OPS = {"sphere": 2, "ellipsoid": 3, "rastrigin": 19, "rosenbrock": 8, "ackley": 18}
PHILOX_OPS = 80               # per Philox-4x32-10 block: 10 rounds x (2 products, 4 xors, 2 adds)


def op_counts(p, prec):
    """Algorithmic operations per particle-variable update, by pipe: the
    Philox blocks (80 integer operations each), the Eq. 2.1 selection (3
    compares + select, integer), the fresh-value map (4 operations at rate
    1 - Cw, FP32 or FP64 by lattice) and the fitness term (FP32 or FP64 by
    precision); a rotated function adds its row of z = M (x - o): D fused
    multiply-adds per variable."""
    base = p["fn"].replace("rot_", "")
    rot = p["D"] if p["fn"].startswith("rot_") else 0
    fresh = 4.0 * (1.0 - p["Cw"])
    c = {"philox_blocks": philox_blocks_per_update(p), "int": 4.0, "fp32": 0.0, "fp64": 0.0}
    c["fp32" if p["lattice"] == "f32" else "fp64"] += fresh
    if prec == "f32":
        c["fp32"] += FIT32_OPS[base] + rot
    else:
        c["fp64"] += FIT64_OPS[base] + rot
    return c


def alu_ops_per_update(p, prec="f32"):
    c = op_counts(p, prec)
    return PHILOX_OPS * c["philox_blocks"] + c["int"] + c["fp32"] + c["fp64"]


def alu_roofline(problems, t, prec, kernel_s, peaks, kernel):
    """Roofline of a generation kernel bound by arithmetic, against the
    measured pipe rates of this GPU (psso_microbench): the shortest time the
    work can take is the largest of Philox blocks / measured Philox rate,
    FP32 operations / measured FP32 FMA rate, FP64 operations / measured FP64
    FMA rate and all operations / issue rate (128 lanes per SM and clock at
    the measured SM clock).  peak = operations / that time, so frac = that
    time / the kernel's time."""
    tot = {"philox_blocks": 0.0, "int": 0.0, "fp32": 0.0, "fp64": 0.0}
    for p in problems:
        u = p["N"] * p["D"] * t
        for k, v in op_counts(p, prec).items():
            tot[k] += v * u
    ops = PHILOX_OPS * tot["philox_blocks"] + tot["int"] + tot["fp32"] + tot["fp64"]
    issue = peaks["sms"] * LANES_PER_SM * peaks["sm_clock_mhz"] * 1e6
    times = {"philox": tot["philox_blocks"] / peaks["philox_blocks_per_s"],
             "fp32": tot["fp32"] / peaks["fp32_fma_per_s"],
             "fp64": tot["fp64"] / peaks["fp64_fma_per_s"],
             "issue": ops / issue}
    limiter = max(times, key=times.get)
    t_roof = times[limiter]
    upd = sum(p["N"] * p["D"] for p in problems) * t
    return {"bound": "alu", "achieved": ops / kernel_s / 1e12, "peak": ops / t_roof / 1e12,
            "unit": "Tops/s", "frac": t_roof / kernel_s, "limiter": limiter,
            "kernel": kernel, "kernel_ms_per_launch": kernel_s * 1e3,
            "ops_per_update": ops / upd, "roofline_ms": t_roof * 1e3,
            "pipe_ms": {k: v * 1e3 for k, v in times.items()},
            "peak_note": "measured by psso_microbench in this run (Philox-4x32-10 blocks, FP32 / FP64 "
                         "FMA chains, SM clock); achieved counts algorithmic operations"}


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_baseline(problems, t_full, seconds):
    """The CPU oracle (as it stands) on all host cores for a bounded sample:
    the first t_s generations of the workload, t_s sized to ~`seconds`."""
    import oracle
    threads = max(1, os.cpu_count() or 1)
    p = problems[0]

    def run(t):
        t0 = time.perf_counter()
        oracle.run_problem(p, t, nthreads=threads)
        return time.perf_counter() - t0

    probe = run(2)
    per_gen = max(probe / 3.0, 1e-6)
    t_s = int(max(2, min(t_full, seconds / per_gen)))
    el = run(t_s)
    upd = p["N"] * p["D"] * t_s
    return {"value": upd / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{p['fn']} N={p['N']} D={p['D']}: initial population + first {t_s} "
                      f"generations in FP64, {threads} OpenMP threads, {el:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workload
    cfg = workload.config(args.workload)
    p = cfg["problems"][0]
    threads = max(1, os.cpu_count() or 1)
    t_full = args.generations or cfg["t"]
    # size one step to ~ (budget / steps) seconds of CPU work
    budget = min(120.0, 8.0 * max(1, args.steps))

    def one(t):
        t0 = time.perf_counter()
        oracle.run_problem(p, t, nthreads=threads)
        return time.perf_counter() - t0

    per_gen = max(one(2) / 3.0, 1e-6)
    t_s = int(max(1, min(t_full, budget / max(1, args.steps) / per_gen)))
    for _ in range(args.warmup):
        one(1)
    times = [one(t_s) for _ in range(args.steps)]
    upd = p["N"] * p["D"] * t_s
    value = upd * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": p["N"], "D": p["D"], "t": t_s,
                       "note": "each step is a bounded sample of the workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"first {t_s} generations per step, {threads} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Replicas on N GPUs: every rank runs the same workload on its own Philox
# streams (no collective on the data path); only the step time is reduced.
def replica_problems(problems, rank):
    """The workload's problems for one rank: instance k of rank r draws from
    Philox stream k + r * count, so no two instances of the job share draws."""
    count = len(problems)
    return [dict(p, sid=int(p["sid"]) + rank * count) for p in problems]


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step, steps, world, max_total_ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_step * steps * world / (max_total_ms / 1e3)


# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of
# the kernel as it stands, keyed by (kernel, workload); each entry carries the
# digest of the kernel's sources at capture time and is reported only while
# the sources still match (a changed kernel reports traffic null).
TRAFFIC = {
    ("rot_gemm_fit", "rotated_d1000"): ("0b1474d8c773c520", 75.650048e6 + 2.041344e6),
    ("sso_generations", "rastrigin_d100"): ("c5a611e6e84c4e41", 1.407488e6 + 0.055552e6),
    ("bat_stream", "batched_512"): ("b96e79894cdf97df", 668.860928e6 + 913.625856e6),
}
_COMMON = ["sso_common.cuh", "devmath.cuh", "psso_internal.h", "checked.cuh"]
KERNEL_SOURCES = {
    "rot_gemm_fit": ["tc_gemm.cuh", "rot_pipeline.cu", "rot_pipeline.h", *_COMMON],
    "sso_generations": ["sso_kernel.cuh", "gen_variant.cu", *_COMMON],
    "bat_stream": ["bat_stream.cuh", "sso_kernel.cuh", "gen_variant.cu", *_COMMON],
}


def source_digest(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2110_01470_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_of(kernel, workload):
    digest, nbytes = TRAFFIC.get((kernel, workload), ("", None))
    return nbytes if digest and digest == source_digest(kernel) else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


REFINE_KERNELS = ("z32", "fix32", "z64", "fix64", "z64_argmin", "fix64_argmin")


def tensor_roofline(psso, problems, prec, sptr, workload, t_gens, gens=20):
    """Rotated swarms on the tensor-core pipeline: per-kernel event timing of
    the first such instance (psso_time_kernels) and the roofline of the GEMM
    kernel.  Algorithmic work is z = M (x - o): 2 N D^2 flops per generation;
    the kernel executes ten BF16 slice products (four 7-bit integer slices per
    operand, weights 0..3, in four exact accumulators) over the padded
    extents.  Each instance is timed early (generations gens+1 .. 2 gens,
    many close decisions) and again around generation t_gens / 2; the share of
    the refinement and FP64 kernels in a generation is reported for both."""
    rot = [p for p in problems if p["fn"].startswith("rot_") and p["N"] >= 128 and p["D"] >= 32]
    if prec != "f32" or not rot:
        return None
    per_instance = []
    for q in rot:
        h = psso.psso_create_ex([q], prec, stream=sptr)
        try:
            psso.psso_run(h, gens)
            early = psso.psso_time_kernels(h, 0, gens)
            late_at = max(t_gens // 2, 3 * gens)
            psso.psso_run(h, late_at - 2 * gens)
            late = psso.psso_time_kernels(h, 0, gens)
            share = {k: sum(v for n, v in ms.items() if n in REFINE_KERNELS) / sum(ms.values())
                     for k, ms in (("early", early), ("late", late))}
            per_instance.append({"fn": q["fn"], "kernels_ms": early, "kernels_ms_late": late,
                                 "late_generation": late_at, "refine_share": share})
        finally:
            psso.psso_destroy(h)
    p = rot[0]
    ms = per_instance[0]["kernels_ms"]
    N, D = p["N"], p["D"]
    Np, Jp, Kp = -(-N // 128) * 128, -(-D // 64) * 64, -(-D // 64) * 64
    t = ms["gemm_fit"] / 1e3
    peaks, which = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    achieved = 2.0 * N * D * D / t / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic_of("rot_gemm_fit", workload),
            "traffic_algorithmic": 2 * 4 * (Np + Jp) * Kp,
            "kernel": "rot_gemm_fit (tcgen05 exact integer-slice GEMM + fitness epilogue)",
            "kernel_ms_per_launch": ms["gemm_fit"],
            "executed_tflops": 10 * 2.0 * Np * Jp * Kp / t / 1e12,
            "peak_note": f"bf16 sustained {which} (kernel timed inside the generation sequence); "
                         "achieved counts 2 N D^2 algorithmic flops, executed_tflops the ten "
                         "BF16 slice products over padded extents",
            "kernels_ms": ms, "instance": {"fn": p["fn"], "N": N, "D": D},
            "per_instance": per_instance}


def accept_rate(psso, problems, prec, t, sptr, stride=10):
    """Mean pBest accept rate alpha per instance over a plain run of t
    generations (from the per-generation log, every `stride`-th generation)."""
    h = psso.psso_create_ex(problems, prec, stream=sptr, log_stride=stride,
                            log_capacity=t // stride + 2)
    try:
        psso.psso_run(h, t)
        out = []
        for k, p in enumerate(problems):
            log = psso.psso_get_log(h, k)
            sel = log["generation"] > 0
            acc = log["accepted"][sel]
            out.append(float(acc.mean()) / p["N"] if acc.size else 0.0)
        return out
    finally:
        psso.psso_destroy(h)


def batched_roofline(psso, problems, prec, t, sptr, live, workload, gens=20):
    """Batched pipeline: per-kernel event timing (psso_time_kernels) and the
    HBM roofline of the dominant step kernel.  Algorithmic bytes per update
    (FP32 positions): write x 4, read the selected source 2 (x with
    probability Cw - Cp, pBest Cp - Cg: 0.2 + 0.3 of 4 bytes), write the pBest
    row 4 alpha -> 6 + 4 alpha; sector-granular compulsory traffic reads x and
    P whole: 12 + 4 alpha.  The whole step's bound is the larger of all bytes /
    HBM and all operations / the measured ALU rate (instances run
    concurrently, so their times do not add)."""
    alpha = accept_rate(psso, problems, prec, t, sptr)
    peaks, which = measured_peaks()
    h = psso.psso_create_ex(problems, prec, stream=sptr)
    try:
        psso.psso_run(h, 3)
        ms = psso.psso_time_batch_kernels(h, gens)
    finally:
        psso.psso_destroy(h)
    stream_upd = step_upd = 0.0
    b_alg = {"stream": 0.0, "step": 0.0}
    b_cmp = {"stream": 0.0, "step": 0.0}
    for p, a in zip(problems, alpha):
        u = p["N"] * p["D"]
        kind = "stream" if (p["D"] > 128 and not p["fn"].startswith("rot_")) else "step"
        b_alg[kind] += u * (6.0 + 4.0 * a)
        b_cmp[kind] += u * (12.0 + 4.0 * a)
        if kind == "stream":
            stream_upd += u
        else:
            step_upd += u
    hbm = peaks["hbm_gbs"] * 1e9
    dom = "stream" if ms["stream"] >= ms["step"] else "step"
    t_dom = ms[dom] / 1e3
    ops_all = sum(alu_ops_per_update(p, prec) * p["N"] * p["D"] for p in problems)
    alu = alu_roofline(problems, 1, prec, 1.0, live, "")
    alu_rate = alu["peak"] * 1e12
    gen_s = (ms["stream"] + ms["step"] + ms["argmin"]) / 1e3
    t_all = max((b_alg["stream"] + b_alg["step"]) / hbm, ops_all / alu_rate)
    t_all_c = max((b_cmp["stream"] + b_cmp["step"]) / hbm, ops_all / alu_rate)
    # the survey's sum over instances of max(bytes / HBM, ops / ALU), for reference
    t_sum_max = sum(max(p["N"] * p["D"] * (6.0 + 4.0 * a) / hbm,
                        alu_ops_per_update(p, prec) * p["N"] * p["D"] / alu_rate)
                    for p, a in zip(problems, alpha))
    return {"bound": "hbm", "achieved": b_alg[dom] / t_dom / 1e9, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": b_alg[dom] / t_dom / hbm,
            "traffic": traffic_of("bat_stream", workload) if dom == "stream" else None,
            "kernel": "bat_stream (batched step kernel, rows over 128 variables)" if dom == "stream"
                      else "bat_step (batched step kernel, rows up to 128 variables)",
            "kernel_ms_per_launch": ms[dom],
            "bytes_per_update_algorithmic": b_alg[dom] / (stream_upd if dom == "stream" else step_upd),
            "achieved_compulsory_gbs": b_cmp[dom] / t_dom / 1e9,
            "frac_compulsory": b_cmp[dom] / t_dom / hbm,
            "kernels_ms_per_generation": ms,
            "generation_ms": gen_s * 1e3,
            "generation_frac": t_all / gen_s, "generation_frac_compulsory": t_all_c / gen_s,
            "generation_frac_sum_of_instance_max": t_sum_max / gen_s,
            "alpha_mean": float(sum(alpha) / len(alpha)),
            "peak_note": f"HBM copy bandwidth {which}; achieved counts 6 + 4 alpha "
                         "algorithmic bytes per update of the kernel's rows (alpha measured per "
                         "instance); the generation fractions bound the whole step"}


def fitness_error(psso, h, problems, prec, sample=64, seed=7):
    """Relative error of the FP32 fitness against FP64 on the final state of
    a run: the stored pBest values (what the run keeps and reports) and a raw
    FP32 evaluation of the same rows, on the gBest and `sample` random
    particles of each instance.  The FP64 values come from psso_evaluate in
    FP64 (the oracle's summation order)."""
    import numpy as np
    if prec != "f32":
        return None
    rng = np.random.default_rng(seed)
    stored, raw = [], []
    for k, p in enumerate(problems[:8]):
        N, D = p["N"], p["D"]
        X, P, pF = psso.psso_get_state(h, k, N, D)
        _, b, _ = psso.psso_best(h, k)
        idx = np.unique(np.concatenate([[b], rng.choice(N, size=min(sample, N), replace=False)]))
        rows = P[idx]
        f64, _ = psso.psso_evaluate(p["fn"], rows, p["o"], p["w"], p["M"], precision="f64")
        f32, _ = psso.psso_evaluate(p["fn"], rows, p["o"], p["w"], p["M"], precision="f32")
        floor = 1e-6 * (20 + np.e) if p["fn"].endswith("ackley") else 0.0
        scale = np.maximum(np.abs(f64), floor)
        scale = np.where(scale > 0, scale, 1.0)
        stored.append(np.abs(pF[idx] - f64) / scale)
        raw.append(np.abs(f32 - f64) / scale)
    stored, raw = np.concatenate(stored), np.concatenate(raw)
    return {"pbest_rel_max": float(stored.max()), "pbest_rel_median": float(np.median(stored)),
            "eval_rel_max": float(raw.max()), "eval_rel_median": float(np.median(raw)),
            "rows": int(stored.size), "target": 1e-6,
            "note": "relative to max(|f64|, 1e-6 (20 + e)) for Ackley, |f64| otherwise"}


def psso_best_values(psso, problems, prec, t, sptr):
    """gBest value of every instance after one plain run of t generations."""
    h = psso.psso_create_ex(problems, prec, stream=sptr)
    try:
        psso.psso_run(h, t)
        return [psso.psso_best(h, k)[0] for k in range(len(problems))]
    finally:
        psso.psso_destroy(h)


def polish_arm(psso, torch, problems, prec, t, pol, sptr, stream, steps, flush):
    """SSO with the gBest polish every K generations (each instance), timed
    with the polish inside the timed region (it synchronises, so the time is
    host wall-clock around device-synchronised steps)."""
    K, n_steps, lr = int(pol["K"]), int(pol["steps"]), float(pol["lr"])
    h = psso.psso_create_ex(problems, prec, stream=sptr)
    times, improved = [], 0
    try:
        for s in range(steps + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            psso.psso_reset(h)
            done, imp = 0, 0
            while done < t:
                c = min(K, t - done)
                psso.psso_run(h, c)
                done += c
                if done % K == 0:
                    for k in range(len(problems)):
                        imp += psso.psso_polish(h, k, n_steps, lr)
            psso.psso_sync(h)
            if s > 0:                   # the first pass is the warm-up
                times.append(time.perf_counter() - t0)
                improved = imp
        on = [psso.psso_best(h, k)[0] for k in range(len(problems))]
    finally:
        psso.psso_destroy(h)
    upd = sum(p["N"] * p["D"] for p in problems) * t
    return {"K": K, "steps": n_steps, "lr": lr, "ms_per_step": 1e3 * sum(times) / len(times),
            "value": upd * len(times) / sum(times), "unit": UNIT,
            "polishes_per_step": (t // K) * len(problems), "improved_per_step": improved,
            "gbest_on": on}


def grad_arm(psso, torch, problems, stream, flush, reps=20):
    """FP32 forward and backward fitness kernels on N random rows per
    problem: device time per call (CUDA events, L2 flushed before each) and
    throughput against the HBM copy peak (bytes: forward reads X, backward
    reads X and writes grad_X; the row-vector and M reads are not counted)."""
    out = []
    for p in problems:
        N, D = p["N"], p["D"]
        g = torch.Generator(device="cuda").manual_seed(7)
        X = (torch.rand((N, D), generator=g, device="cuda") * (p["ub"] - p["lb"]) + p["lb"])
        o = torch.tensor(p["o"], dtype=torch.float32, device="cuda")
        w = None if p["w"] is None else torch.tensor(p["w"], dtype=torch.float32, device="cuda")
        M = None if p["M"] is None else torch.tensor(p["M"], dtype=torch.float32, device="cuda")
        f = torch.empty(N, device="cuda")
        gf = torch.ones(N, device="cuda")
        gX = torch.empty_like(X)
        ptr = lambda a: None if a is None else a.data_ptr()
        sp = stream.cuda_stream
        # the *_ws calls: rotated products on the tensor cores (the rest: warp kernels)
        nws = psso.psso_fitness_workspace_size(p["fn"], N, D)
        ws = torch.empty(max(nws, 1), dtype=torch.uint8, device="cuda")

        def fwd():
            psso.psso_fitness_forward_ws(p["fn"], N, D, X.data_ptr(), o.data_ptr(), ptr(w), ptr(M),
                                         f.data_ptr(), ws.data_ptr(), nws, sp)

        def bwd():
            psso.psso_fitness_backward_ws(p["fn"], N, D, X.data_ptr(), o.data_ptr(), ptr(w),
                                          ptr(M), gf.data_ptr(), gX.data_ptr(), ws.data_ptr(), nws,
                                          sp)

        res = {"fn": p["fn"], "N": N, "D": D, "tensor_cores": nws > 0}
        for name, call, nbytes in (("forward", fwd, 4 * N * D), ("backward", bwd, 8 * N * D)):
            call()
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            m = statistics.median(ms)
            res[name] = {"ms": m, "rows_per_s": N / (m / 1e3), "gbs": nbytes / (m / 1e3) / 1e9}
            if p["fn"].startswith("rot_"):
                mult = 1 if name == "forward" else 2
                res[name]["gemm_tflops_algorithmic"] = mult * 2.0 * N * D * D / (m / 1e3) / 1e12
        out.append(res)
    return out


def sptr_of(torch):
    return torch.cuda.current_stream().cuda_stream


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2110_01470_gb300.build import build_library
    build_library()
    import paper_2110_01470_gb300 as psso
    import workload

    live = psso.psso_microbench(sptr_of(torch))   # measured pipe / latency peaks of this GPU
    cfg = workload.config(args.workload)
    t = args.generations or cfg["t"]
    problems = replica_problems(cfg["problems"], rank)
    prec = cfg["precision"]
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    upd_per_step = sum(p["N"] * p["D"] for p in problems) * t
    evals_per_step = sum(p["N"] for p in problems) * (t + 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    timed_launches = [0]

    def timed_steps(h, steps, warm, gens=None):
        gens = gens or t
        for _ in range(warm):
            psso.psso_reset(h)
            psso.psso_run(h, gens)
        psso.psso_sync(h)
        step_ms, kern_ms = [], []
        launches0 = psso.psso_stats(h)["launches"]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            psso.psso_reset(h)
            e1.record(stream)
            psso.psso_run(h, gens)
            e2.record(stream)
            e2.synchronize()
            step_ms.append(e0.elapsed_time(e2))
            kern_ms.append(e1.elapsed_time(e2))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        psso.psso_sync(h)
        timed_launches[0] = psso.psso_stats(h)["launches"] - launches0
        return step_ms, kern_ms

    def tuned_shape(precision):
        """Launch shape from the library's autotuner (cached per process)."""
        if args.threads_per_block or not args.autotune:
            return {"threads_per_block": args.threads_per_block}, None
        return psso.psso_autotune(problems, precision, generations=min(t, 200), stream=sptr)

    # --- main arm: the workload's precision -------------------------------------------
    shape, tune_report = tuned_shape(prec)
    h = psso.psso_create_ex(problems, prec, stream=sptr, **shape)
    st = psso.psso_stats(h)
    with ClockSampler(local) as clk:
        step_ms, kern_ms = timed_steps(h, args.steps, args.warmup)
    launches_main = timed_launches[0]
    st_end = psso.psso_stats(h)
    rechecks, refinements = st_end["rechecks"], st_end["refinements"]
    best = psso.psso_best(h, 0)
    fit_err = fitness_error(psso, h, problems, prec)
    psso.psso_destroy(h)
    total = sum(step_ms)
    total = max_over_ranks(total, dist, "cuda")
    value = job_rate(upd_per_step, args.steps, world, total)
    evals = job_rate(evals_per_step, args.steps, world, total)

    # --- FP64-fitness arm on the same workload ------------------------------------------
    fp64 = None
    if prec != "f64" and args.fp64_steps > 0:
        shape64, _ = tuned_shape("f64")
        h = psso.psso_create_ex(problems, "f64", stream=sptr, **shape64)
        # a bounded sample where FP64 is slow (rotated swarms: GB300's FP64 rate):
        # the first t64 generations, sized to about 3 s per step
        g_probe = min(t, 10)
        p_ms, _ = timed_steps(h, 1, 0, g_probe)
        t64 = int(min(t, max(g_probe, 3000.0 / max(p_ms[0] / g_probe, 1e-6))))
        s64, k64 = timed_steps(h, args.fp64_steps, 1, t64)
        b64 = psso.psso_best(h, 0)
        psso.psso_destroy(h)
        v64 = upd_per_step * (t64 / t) * len(s64) / (sum(s64) / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": sum(s64) / len(s64),
                "kernel_ms": sum(k64) / len(k64), "generations": t64,
                "speedup_f32_over_f64": value / world / v64,
                "same_gbest": bool(b64[1] == best[1] and b64[0] == best[0]) if t64 == t else None}

    # --- opt-in gBest polish (workloads that name one) -------------------------------------
    polish = None
    if cfg.get("polish") and args.polish_steps > 0:
        polish = polish_arm(psso, torch, problems, prec, t, cfg["polish"], sptr, stream,
                            args.polish_steps, flush)
        polish["gbest_off"] = psso_best_values(psso, problems, prec, t, sptr)
    grad = None
    if cfg.get("polish"):
        grad = grad_arm(psso, torch, problems, stream, flush)

    # --- end to end through the public API with host buffers ------------------------------
    e2e_t, h2d, d2h = [], 0, 0
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        shape_e, _ = tuned_shape(prec)        # the user's call; answered from the cache
        h = psso.psso_create_ex(problems, prec, stream=sptr, **shape_e)
        psso.psso_run(h, t)
        v, i, row = psso.psso_best(h, 0, problems[0]["D"])
        s = psso.psso_stats(h)
        psso.psso_destroy(h)
        torch.cuda.synchronize()
        if k > 0:                       # the first call pays one-time module loading
            e2e_t.append(time.perf_counter() - t0)
            h2d, d2h = s["h2d_bytes"], s["d2h_bytes"]
    e2e_value = upd_per_step * len(e2e_t) / sum(e2e_t) * world if e2e_t else None

    # --- roofline of the dominant kernel ------------------------------------------------------
    p0 = problems[0]
    kernel_s = (sum(kern_ms) / len(kern_ms)) / 1e3
    n_bat = st.get("batch_classes", 0)
    if n_bat and st["blocks"] == 0:
        roofline = batched_roofline(psso, problems, prec, t, sptr, live, args.workload)
    else:
        roofline = tensor_roofline(psso, problems, prec, sptr, args.workload, t)
    if roofline is None:
        per_lane = -(-(-(-p0["D"] // 4)) // 32)          # chunks of 4 variables per lane
        width = 1 if per_lane <= 1 else 2 if per_lane <= 2 else 4 if per_lane <= 4 else 8
        name = (f"sso_generations<{'float' if p0['lattice'] == 'f32' else 'double'}, "
                f"F32R={1 if prec == 'f32' else 0}, MC={width}>")
        roofline = alu_roofline(problems, t, prec, kernel_s, live, name)
        roofline["traffic"] = (traffic_of("sso_generations", args.workload)
                               if len(problems) == 1 else None)
        # the sequential generations also bound the run from below by latency:
        # at least one store -> polled-load hand-off per generation across blocks
        roofline["latency_floor_ms"] = t * live["l2_handoff_ns"] * 1e-6 if st["blocks"] > 1 else None
        roofline["us_per_generation"] = kernel_s * 1e6 / t

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "f32" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "fn": p0["fn"], "N": p0["N"], "D": p0["D"],
                   "t": t, "precision": "f32+f64 recheck" if prec == "f32" else "f64",
                   "lattice": p0["lattice"], "instances_per_gpu": len(problems),
                   "blocks": st["blocks"], "threads_per_block": st["threads_per_block"],
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (256 MiB write outside the timed steps)"},
        "fitness_evals_per_s": evals,
        "gpu_launches": launches_main,
        "rechecks_last_step": rechecks,
        "refinements_last_step": refinements,
        "gbest": {"value": best[0], "index": best[1]},
        "fp64": fp64,
        "autotune": tune_report,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roofline,
        "fitness_err_vs_fp64": fit_err,
        "peaks": live,
        "clocks": clk.summary(),
    }
    if polish is not None:
        line["polish"] = polish
    if grad is not None:
        line["fitness_grad"] = grad
    if world == 1 or rank == 0:
        line["cpu_baseline"] = cpu_baseline(problems, t, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
