"""Seeded synthetic problem data for SSO runs.

This module makes the *data* that defines a benchmark problem -- shift vectors
o, orthogonal rotation matrices M, ellipsoid weights w, and the table of
independent instances of a batched run -- and the five named workloads.  It
holds none of the SSO method's arithmetic (no stepwise update, no fitness, no
Philox draws of the method): the oracle-side tests and the CUDA-side bench both
consume these arrays as inputs.  Only numpy is used.

Workloads (the test functions are those of Table 3.2 of the paper, in shifted
or rotated form; sizes are the synthetic configurations this library is
measured on):
  sphere_d30     shifted sphere, D=30, N=100, t=1000, [-100,100], o~U[-80,80]^D,
                 FP64 lattice, Cg/Cp/Cw = 0.4/0.7/0.9, seed 1
  rastrigin_d100 shifted Rastrigin, D=100, N=1024, t=5000, [-5.12,5.12],
                 o~U[-4,4]^D (float-exact), FP32 lattice
  rotated_d1000  rotated ellipsoid / Rastrigin, D=1000, N=8192, t=2000,
                 [-100,100], M Haar-orthogonal (QR of a Gaussian, FP64)
  batched_512    512 independent instances, D ~ log-uniform int [10,1000],
                 N ~ log-uniform int [64,4096], function uniform over
                 {sphere, Rastrigin, Rosenbrock, Ackley}, t=1000
  grad_d256      Rosenbrock and rotated Ackley, D=256, N=4096, t=3000
  paper_rosenbrock_n{100,200,300,350}
                 the paper's timing workload (Table 3.10): Rosenbrock, D=50,
                 t=1000, bounds [-2.048, 2.048], no shift, FP64, and the
                 paper's interval triple Cw/Cp/Cg = 0.3/0.6/0.8 in the interval
                 order Eq. 2.1 prints (keep, pBest, gBest, fresh)
"""
from __future__ import annotations

import math

import numpy as np

# Stream tags so that the data of one seed never reuses another array's stream.
_TAG_SHIFT, _TAG_ROT, _TAG_TABLE = 0x5348, 0x524F, 0x5441

# Search bounds of Table 3.2 for the four batched functions.
BOUNDS = {
    "sphere": (-100.0, 100.0),
    "ellipsoid": (-100.0, 100.0),
    "rastrigin": (-5.12, 5.12),
    "rosenbrock": (-2.048, 2.048),
    "ackley": (-32.768, 32.768),
    "rot_ellipsoid": (-100.0, 100.0),
    "rot_rastrigin": (-5.12, 5.12),
    "rot_ackley": (-32.768, 32.768),
    "hyper_ellipsoid": (-5.12, 5.12),
    "schwefel12": (-65.536, 65.536),
    "griewank": (-600.0, 600.0),
    "powell": (-4.0, 5.0),
    # Table 3.2 prints [-5.12, 5.12]; the function's minimum (z_j = 420.9687)
    # lies in the usual [-500, 500]
    "schwefel": (-500.0, 500.0),
}


def _rng(seed: int, tag: int, extra: int = 0) -> np.random.Generator:
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, (tag << 32) | (extra & 0xFFFFFFFF)],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def shift(D: int, lo: float, hi: float, seed: int, lattice: str = "f64", stream: int = 0):
    """Shift vector o ~ U[lo, hi]^D.  With the FP32 lattice every entry is rounded
    to the nearest float so that FP32 and FP64 evaluations see the same o."""
    o = _rng(seed, _TAG_SHIFT, stream).uniform(lo, hi, D)
    if lattice == "f32":
        o = o.astype(np.float32).astype(np.float64)
    return np.ascontiguousarray(o, dtype=np.float64)


def rotation(D: int, seed: int, stream: int = 0):
    """Haar-random orthogonal D x D matrix (FP64): QR of a standard Gaussian
    matrix, columns sign-fixed by the diagonal of R."""
    A = _rng(seed, _TAG_ROT, stream).standard_normal((D, D))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))[None, :]
    return np.ascontiguousarray(Q, dtype=np.float64)


def ellipsoid_weights(D: int):
    """w_j = 10^(6 j / (D-1)), j = 0..D-1 (w = 1 for D = 1)."""
    if D == 1:
        return np.ones(1, dtype=np.float64)
    j = np.arange(D, dtype=np.float64)
    return np.power(10.0, 6.0 * j / (D - 1))


def problem(fn: str, N: int, D: int, *, seed: int = 1, lattice: str = "f64",
            shift_range=None, bounds=None, Cg=0.4, Cp=0.7, Cw=0.9, stream: int = 0,
            order: str = "gpx"):
    """A complete problem description (plain dict of data) for one SSO instance.
    ``order`` is the interval order of Eq. 2.1: "gpx" (gBest, pBest, keep with
    Cg <= Cp <= Cw) or "paper" (keep, pBest, gBest with Cw <= Cp <= Cg)."""
    lb, ub = bounds if bounds is not None else BOUNDS[fn]
    if shift_range is None:
        shift_range = (0.8 * lb, 0.8 * ub)
    o = shift(D, shift_range[0], shift_range[1], seed, lattice, stream)
    w = ellipsoid_weights(D) if fn in ("ellipsoid", "rot_ellipsoid") else None
    M = rotation(D, seed, stream) if fn.startswith("rot_") else None
    return dict(fn=fn, N=N, D=D, lb=lb, ub=ub, Cg=Cg, Cp=Cp, Cw=Cw, seed=seed,
                sid=stream, lattice=lattice, order=order, o=o, w=w, M=M)


def batched_table(count: int = 512, seed: int = 1, lattice: str = "f32"):
    """Independent instances of a batched run: D ~ floor(exp U[ln 10, ln 1001)),
    N ~ floor(exp U[ln 64, ln 4097)), function uniform over the four separable
    test functions, bounds of Table 3.2, shift o ~ U[0.8 lb, 0.8 ub]^D.
    Instance k uses Philox stream k of the run seed."""
    r = _rng(seed, _TAG_TABLE)
    Ds = np.floor(np.exp(r.uniform(math.log(10), math.log(1001), count))).astype(np.int64)
    Ns = np.floor(np.exp(r.uniform(math.log(64), math.log(4097), count))).astype(np.int64)
    fns = r.integers(0, 4, count)
    names = ["sphere", "rastrigin", "rosenbrock", "ackley"]
    out = []
    for k in range(count):
        out.append(problem(names[fns[k]], int(Ns[k]), int(Ds[k]), seed=seed,
                           lattice=lattice, stream=k))
    return out


def config(name: str):
    """The named synthetic workloads (see the module docstring)."""
    if name == "sphere_d30":
        p = problem("sphere", 100, 30, seed=1, lattice="f64", shift_range=(-80.0, 80.0))
        return dict(problems=[p], t=1000, precision="f64")
    if name == "rastrigin_d100":
        p = problem("rastrigin", 1024, 100, seed=1, lattice="f32", shift_range=(-4.0, 4.0))
        return dict(problems=[p], t=5000, precision="f32")
    if name == "rotated_d1000":
        ps = [problem(f, 8192, 1000, seed=1, lattice="f32")
              for f in ("rot_ellipsoid", "rot_rastrigin")]
        return dict(problems=ps, t=2000, precision="f32")
    if name == "batched_512":
        return dict(problems=batched_table(512, seed=1), t=1000, precision="f32")
    if name == "grad_d256":
        ps = [problem(f, 4096, 256, seed=1, lattice="f32") for f in ("rosenbrock", "rot_ackley")]
        return dict(problems=ps, t=3000, precision="f32", polish=dict(K=50, steps=20, lr=1e-3))
    if name.startswith("paper_rosenbrock_n"):
        N = int(name[len("paper_rosenbrock_n"):])
        p = problem("rosenbrock", N, 50, seed=1, lattice="f64", shift_range=(0.0, 0.0),
                    Cg=0.8, Cp=0.6, Cw=0.3, order="paper")
        return dict(problems=[p], t=1000, precision="f64")
    raise KeyError(name)
