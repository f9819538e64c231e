"""Builds ``libpsso.so`` (the CUDA library behind include/psso.h) in-tree.

Every ``csrc/*.cu`` translation unit is compiled by nvcc for sm_103a in
parallel (``gen_variant.cu`` once per kernel variant and width), then linked
into one shared library next to this file.  Usage:
``python -m paper_2110_01470_gb300.build`` or ``build_library()``.

``build_library(trace=True)`` (or ``--trace``) builds a profiling copy instead:
the same sources compiled with ``-DPSSO_TRACE`` (the persistent kernel then
stamps ``%globaltimer`` at its phase boundaries, see ``trace_generations``)
into ``_build/libpsso_trace.so``; the package's own library is untouched.
``build_library(checked=True)`` (or ``--checked``) builds the index-checked
copy ``_build/libpsso_checked.so`` (``-DPSSO_CHECKED``: every kernel verifies
the indices it computes before the access and records the first failure,
read back with ``psso_check_report``).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build", "psso")
LIB = os.path.join(HERE, "libpsso.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libpsso.so")
    return cand


def _newest_input() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(f) for f in files)


TRACE_OBJDIR = os.path.join(ROOT, "_build", "trace")
TRACE_LIB = os.path.join(ROOT, "_build", "libpsso_trace.so")
CHECKED_OBJDIR = os.path.join(ROOT, "_build", "checked")
CHECKED_LIB = os.path.join(ROOT, "_build", "libpsso_checked.so")


def build_library(force: bool = False, verbose: bool = False, trace: bool = False,
                  checked: bool = False) -> str:
    """Compile and link libpsso.so if any source is newer than it (with
    ``trace``: the phase-stamped profiling copy in ``_build/``; with
    ``checked``: the index-checked copy in ``_build/``)."""
    if trace and checked:
        raise ValueError("build either the traced or the checked copy")
    lib = TRACE_LIB if trace else CHECKED_LIB if checked else LIB
    objdir = TRACE_OBJDIR if trace else CHECKED_OBJDIR if checked else OBJDIR
    flags = NVCC_FLAGS + (["-DPSSO_TRACE"] if trace else []) + (["-DPSSO_CHECKED"] if checked else [])
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(objdir, exist_ok=True)
    variant_src = os.path.join(CSRC, "gen_variant.cu")
    jobs = [(src, os.path.basename(src)[:-3], [])
            for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))) if src != variant_src]
    # the persistent kernel: one object per (variant, width), compiled in parallel
    jobs += [(variant_src, f"gen_variant_{v}_{m}", [f"-DPSSO_VARIANT={v}", f"-DPSSO_MC={m}"])
             for v in range(3) for m in (1, 2, 4, 8)]
    # longest first
    jobs.sort(key=lambda j: (j[0] != variant_src, -int(j[1][-1]) if j[0] == variant_src else 0))
    exe = nvcc()

    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    newest_header = max(os.path.getmtime(f) for f in headers)

    def compile_one(job):
        src, name, defs = job
        obj = os.path.join(objdir, name + ".o")
        # an object is current when newer than its source and every header
        if not force and os.path.exists(obj) and \
                os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header):
            return obj
        cmd = [exe, *ARCH, *flags, *defs, "-c", src, "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{p.stderr}")
        if verbose and p.stderr:
            sys.stderr.write(p.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, jobs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True, trace="--trace" in sys.argv,
                        checked="--checked" in sys.argv))
