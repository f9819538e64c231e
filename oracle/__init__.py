"""CPU oracle for Parallel Simplified Swarm Optimization (arXiv 2110.01470).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2110_01470_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``psso_oracle.c`` (plain sequential C, FP64).  This
module compiles it with gcc on first use and exposes thin numpy wrappers.

Parity status per function (how each is pinned, see ``tests/test_oracle_*.py``):
  * ``philox``   -- pinned against Triton's independent Philox-4x32-10
                    (interpreter mode, CPU) and bijectivity of one round.
  * ``fresh``    -- pinned by the closed-form lattice map on Triton's Philox words,
                    range and uniformity tests.
  * ``sinpi`` / ``expm1`` -- pinned against mpmath at 300 bits (<= 2 ulp) and
                    exact special values.
  * ``fitness``  -- pinned by closed forms at hand-computed points (Table 3.2
                    definitions), rotation invariance, and mpmath evaluation.
  * ``run``      -- pinned by special cases that reduce to closed forms
                    (Cg = 1, Cp = 1, Cw = 0), invariants (monotone pBest / gBest,
                    bounds, lattice membership, lowest-index arg-min, binomial
                    branch frequencies) and brute-force grid search at D <= 2.
                    No external trajectory exists to compare whole runs with.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psso_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FN = {
    "sphere": 0,
    "ellipsoid": 1,
    "rastrigin": 2,
    "rosenbrock": 3,
    "ackley": 4,
    "rot_ellipsoid": 5,
    "rot_rastrigin": 6,
    "rot_ackley": 7,
    "hyper_ellipsoid": 8,
    "schwefel12": 9,
    "griewank": 10,
    "powell": 11,
    "schwefel": 12,
}
LATTICE = {"f64": 0, "f32": 1}
TAG_INIT, TAG_RHO, TAG_FRESH = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``psso_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    u32, u64, i64, d, i32 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                             ctypes.c_double, ctypes.c_int)
    vp = ctypes.c_void_p
    lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_rho.argtypes = [u64, u32, u32, u32, u32]
    lib.oracle_rho.restype = u32
    lib.oracle_fresh.argtypes = [i32, u64, u32, u32, u32, u32, u32, d, d]
    lib.oracle_fresh.restype = d
    lib.oracle_sinpi.argtypes = [d]
    lib.oracle_sinpi.restype = d
    lib.oracle_expm1.argtypes = [d]
    lib.oracle_expm1.restype = d
    lib.oracle_fitness.argtypes = [i32, i64, vp, vp, vp, vp]
    lib.oracle_fitness.restype = d
    lib.oracle_run.argtypes = [i32, i32, i64, i64, d, d, d, d, d, u64, u32, vp, vp, vp,
                               i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.oracle_run.restype = i32
    lib.oracle_run_ex.argtypes = [i32, i32, i32, i32, i64, i64, d, d, d, d, d, u64, u32, vp, vp,
                                  vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.oracle_run_ex.restype = i32
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = i32
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def philox(ctr, key):
    """Philox-4x32-10 block for counter ``ctr`` (4 x u32) and key ``key`` (2 x u32)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def rho(seed, sid, g, i, j):
    return int(_load().oracle_rho(seed, sid, g, i, j))


def fresh(lattice, seed, sid, tag, g, i, j, lb, ub):
    return float(_load().oracle_fresh(LATTICE[lattice], seed, sid, tag, g, i, j, lb, ub))


def sinpi(x):
    return float(_load().oracle_sinpi(float(x)))


def expm1(x):
    return float(_load().oracle_expm1(float(x)))


def fitness(fn, x, o=None, w=None, M=None):
    """Fitness of one particle ``x`` (length D) for function ``fn``."""
    lib = _load()
    x = _f64(x)
    D = x.size
    o = _f64(o, D)
    w = _f64(w, D)
    M = _f64(M, D * D)
    return float(lib.oracle_fitness(FN[fn], D, _ptr(x), _ptr(o), _ptr(w), _ptr(M)))


ORDER = {"gpx": 0, "paper": 1}
FLOW = {"sync": 0, "async": 1}


def run(fn, N, D, lb, ub, Cg, Cp, Cw, seed, t, *, lattice="f64", sid=0, o=None, w=None,
        M=None, nthreads=1, order="gpx", flow="sync"):
    """One SSO run of ``t`` generations.  Returns a dict of numpy arrays:
    X, P (N x D), pF (N), G (D), log_b, log_v, log_acc (t+1), branch (4).
    ``order``: "gpx" (intervals gBest, pBest, keep; Cg <= Cp <= Cw) or "paper"
    (Eq. 2.1 as printed: keep, pBest, gBest; Cw <= Cp <= Cg).  ``flow``: "sync"
    (Alg. 2-4) or "async" (Alg. 1, particle by particle)."""
    lib = _load()
    o = _f64(o, D)
    w = _f64(w, D)
    M = _f64(M, D * D)
    X = np.empty((N, D), dtype=np.float64)
    P = np.empty((N, D), dtype=np.float64)
    pF = np.empty(N, dtype=np.float64)
    G = np.empty(D, dtype=np.float64)
    log_b = np.empty(t + 1, dtype=np.int64)
    log_v = np.empty(t + 1, dtype=np.float64)
    log_acc = np.empty(t + 1, dtype=np.int64)
    branch = np.zeros(4, dtype=np.int64)
    rc = lib.oracle_run_ex(FN[fn], LATTICE[lattice], ORDER[order], FLOW[flow], N, D, lb, ub,
                           Cg, Cp, Cw, seed, sid, _ptr(o), _ptr(w), _ptr(M), t, nthreads,
                           _ptr(X), _ptr(P), _ptr(pF), _ptr(G), _ptr(log_b), _ptr(log_v),
                           _ptr(log_acc), _ptr(branch))
    if rc != 0:
        raise ValueError(f"oracle_run rejected its arguments (code {rc})")
    return dict(X=X, P=P, pF=pF, G=G, log_b=log_b, log_v=log_v, log_acc=log_acc,
                branch=branch)


def run_problem(p, t, *, nthreads=1, flow="sync"):
    """``run`` on a problem description (a dict with the keys fn, N, D, lb, ub,
    Cg, Cp, Cw, seed and optional lattice, sid, order, o, w, M)."""
    return run(p["fn"], p["N"], p["D"], p["lb"], p["ub"], p["Cg"], p["Cp"], p["Cw"], p["seed"],
               t, lattice=p.get("lattice", "f64"), sid=p.get("sid", 0), o=p.get("o"),
               w=p.get("w"), M=p.get("M"), nthreads=nthreads, order=p.get("order", "gpx"),
               flow=flow)


def max_threads():
    return int(_load().oracle_max_threads())


def host_description():
    """CPU model and core count of this host (for the CPU-baseline record)."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu": model, "nproc": os.cpu_count()}
