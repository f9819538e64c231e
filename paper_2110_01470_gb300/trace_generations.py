"""Phase timing of the persistent generation kernel (profiling aid).

Builds a separate copy of the library with ``-DPSSO_TRACE`` (the kernel then
stamps ``%globaltimer`` at the phase boundaries of its control warp for
generations 100..163 of the first 160 blocks), runs shifted Rastrigin D=100,
N=1024 with FP32 fitness for 200 generations, and prints the median time of
each phase from the start of a generation, the spread between blocks and the
generation period.  The stamps cost about 0.3 us per generation.

    python -m paper_2110_01470_gb300.trace_generations [threads_per_block]

Phase stamps (control warp of a pipelined block): 0 generation start,
5 records of g-1 complete, 8 their arg-min, 9 gBest row in shared memory,
1 verdict, 2 speculative candidates in, 3 record sent, 4 row published.
"""
from __future__ import annotations

import ctypes
import sys

import numpy as np

from . import build as B

TRACE_BLOCKS, TRACE_GENS, TRACE_POINTS = 160, 64, 12
PHASES = [(5, "records of g-1 complete"), (8, "arg-min of the records"), (9, "gBest row"),
          (1, "verdict"), (2, "speculative candidates in"), (3, "record sent"),
          (4, "row published")]


def build_traced() -> str:
    """Compiles the library with the phase stamps into _build/ (not the package)."""
    return B.build_library(trace=True)


def main(tpb: int = 0) -> None:
    sys.path.insert(0, B.ROOT)
    lib_path = build_traced()
    import paper_2110_01470_gb300 as psso
    import workload
    psso.load(lib_path)
    p = workload.config("rastrigin_d100")["problems"][0]
    h = psso.psso_create_ex([p], "f32", threads_per_block=tpb)
    try:
        st = psso.psso_stats(h)
        psso.psso_run(h, 200)
        psso.psso_sync(h)
        buf = np.zeros((TRACE_BLOCKS, TRACE_GENS, TRACE_POINTS), dtype=np.uint64)
        rc = psso._lib.psso_trace_dump(ctypes.c_void_p(buf.ctypes.data), ctypes.c_size_t(buf.nbytes))
        if rc != 0:
            raise RuntimeError(f"psso_trace_dump failed ({rc})")
    finally:
        psso.psso_destroy(h)
    nb = min(st["blocks"], TRACE_BLOCKS)
    b = buf[:nb, 1:-1].astype(np.int64)            # drop the edge generations
    t0 = b[:, :, 0]
    print(f"blocks {st['blocks']} x {st['threads_per_block']} threads")
    print(f"period: median {np.median(np.diff(t0, axis=1)):.0f} ns")
    for k, name in PHASES:
        d = b[:, :, k] - t0
        print(f"{name:28s} median {np.median(d):7.0f} ns  p90 {np.percentile(d, 90):7.0f} ns")
    sent = b[:, :, 3]
    print(f"record-send spread across blocks: median {np.median(sent.max(0) - sent.min(0)):.0f} ns")
    late = np.bincount(np.argmax(sent, axis=0), minlength=nb)
    print(f"last block to send, most often: rank {int(np.argmax(late))} ({int(late.max())} of {sent.shape[1]})")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
