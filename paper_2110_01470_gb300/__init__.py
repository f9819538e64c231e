"""GB300 (sm_103a) implementation of the hot path of Parallel Simplified Swarm
Optimization (Yeh, Liu, Tan, Huang, arXiv 2110.01470).

This module is a thin ctypes binding over the C ABI of ``include/psso.h``:
the same entry points, with argument marshalling only.  Every step of an SSO
generation (Eq. 2.1 update, fitness, pBest update, gBest arg-min) runs in the
CUDA kernels of ``libpsso.so``; there is no CPU fallback -- importing works
without a GPU, but any call fails loudly if the library is missing.

    import paper_2110_01470_gb300 as psso
    h = psso.psso_create(psso.PSSO_SPHERE, 100, 30, -100, 100, 0.4, 0.7, 0.9, 1)
    psso.psso_run(h, 1000)
    value, index, row = psso.psso_best(h, 0)
    psso.psso_destroy(h)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpsso.so")

# psso_status
PSSO_OK, PSSO_ERR_ARG, PSSO_ERR_CUDA, PSSO_ERR_OOM, PSSO_ERR_TIMEOUT, PSSO_ERR_STATE, \
    PSSO_ERR_UNSUPPORTED = range(7)
# psso_fn
PSSO_SPHERE, PSSO_ELLIPSOID, PSSO_RASTRIGIN, PSSO_ROSENBROCK, PSSO_ACKLEY, \
    PSSO_ROT_ELLIPSOID, PSSO_ROT_RASTRIGIN, PSSO_ROT_ACKLEY, PSSO_HYPER_ELLIPSOID, \
    PSSO_SCHWEFEL12, PSSO_GRIEWANK, PSSO_POWELL, PSSO_SCHWEFEL = range(13)
PSSO_LATTICE_F64, PSSO_LATTICE_F32 = 0, 1
PSSO_PREC_F64, PSSO_PREC_F32_RECHECK = 0, 1
PSSO_ORDER_GPX, PSSO_ORDER_PAPER = 0, 1
PSSO_FLOW_SYNC, PSSO_FLOW_ASYNC = 0, 1

FN = {"sphere": PSSO_SPHERE, "ellipsoid": PSSO_ELLIPSOID, "rastrigin": PSSO_RASTRIGIN,
      "rosenbrock": PSSO_ROSENBROCK, "ackley": PSSO_ACKLEY, "rot_ellipsoid": PSSO_ROT_ELLIPSOID,
      "rot_rastrigin": PSSO_ROT_RASTRIGIN, "rot_ackley": PSSO_ROT_ACKLEY,
      "hyper_ellipsoid": PSSO_HYPER_ELLIPSOID, "schwefel12": PSSO_SCHWEFEL12,
      "griewank": PSSO_GRIEWANK, "powell": PSSO_POWELL, "schwefel": PSSO_SCHWEFEL}
LATTICE = {"f64": PSSO_LATTICE_F64, "f32": PSSO_LATTICE_F32}
PRECISION = {"f64": PSSO_PREC_F64, "f32": PSSO_PREC_F32_RECHECK}
ORDER = {"gpx": PSSO_ORDER_GPX, "paper": PSSO_ORDER_PAPER}

_STATUS_NAMES = {0: "PSSO_OK", 1: "PSSO_ERR_ARG", 2: "PSSO_ERR_CUDA", 3: "PSSO_ERR_OOM",
                 4: "PSSO_ERR_TIMEOUT", 5: "PSSO_ERR_STATE", 6: "PSSO_ERR_UNSUPPORTED"}


class PssoError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class psso_problem(ctypes.Structure):
    _fields_ = [("fn", ctypes.c_int32), ("lattice", ctypes.c_int32), ("N", ctypes.c_int64),
                ("D", ctypes.c_int64), ("lb", ctypes.c_double), ("ub", ctypes.c_double),
                ("Cg", ctypes.c_double), ("Cp", ctypes.c_double), ("Cw", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32),
                ("order", ctypes.c_uint32), ("shift", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("rotation", ctypes.c_void_p)]


class psso_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("single_block_max", ctypes.c_int32), ("log_stride", ctypes.c_int32),
                ("log_capacity", ctypes.c_int64), ("spin_limit", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("max_blocks", ctypes.c_int32),
                ("fault_skip_rank", ctypes.c_int32), ("residency", ctypes.c_int32),
                ("pipeline", ctypes.c_int32), ("tensor_rotation", ctypes.c_int32),
                ("batch_stream", ctypes.c_int32), ("batch_blocks_per_sm", ctypes.c_int32),
                ("flow", ctypes.c_int32)]


class psso_tune_report(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("batch_blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


class psso_peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_per_s", ctypes.c_double), ("fp64_fma_per_s", ctypes.c_double),
                ("int_mad_per_s", ctypes.c_double), ("int_mulhi_xor_per_s", ctypes.c_double),
                ("philox_blocks_per_s", ctypes.c_double), ("l2_handoff_ns", ctypes.c_double),
                ("grid_barrier_ns", ctypes.c_double), ("cluster_barrier_ns", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("sms", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class psso_log_entry(ctypes.Structure):
    _fields_ = [("generation", ctypes.c_int64), ("index", ctypes.c_int64),
                ("value", ctypes.c_double), ("value_lo", ctypes.c_float),
                ("value_hi", ctypes.c_float), ("accepted", ctypes.c_int64),
                ("rechecks", ctypes.c_int64)]


class psso_stats_t(ctypes.Structure):
    _fields_ = [("generations", ctypes.c_int64), ("evaluations", ctypes.c_int64),
                ("updates", ctypes.c_int64), ("rechecks", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("blocks", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("instances", ctypes.c_int32), ("batch_classes", ctypes.c_int32),
                ("refinements", ctypes.c_int64), ("launches", ctypes.c_int64)]


_lib = None


def load(path: str = None):
    """Load libpsso.so (raises if it has not been built).  ``path`` (or the
    environment variable PSSO_LIBRARY) selects another build of the same
    sources, e.g. the index-checked copy of ``build_library(checked=True)``."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PSSO_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2110_01470_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "psso_create": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                         ctypes.c_uint64, ctypes.POINTER(H)], st),
        "psso_create_ex": ([ctypes.POINTER(psso_problem), ctypes.c_int32,
                            ctypes.POINTER(psso_config), ctypes.POINTER(H)], st),
        "psso_run": ([H, ctypes.c_int64], st),
        "psso_sync": ([H], st),
        "psso_reset": ([H], st),
        "psso_best": ([H, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p], st),
        "psso_get_state": ([H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p], st),
        "psso_get_log": ([H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                          ctypes.POINTER(ctypes.c_int64)], st),
        "psso_stats": ([H, ctypes.POINTER(psso_stats_t)], st),
        "psso_generation": ([H], ctypes.c_int64),
        "psso_save": ([H, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], st),
        "psso_load": ([H, ctypes.c_void_p, ctypes.c_size_t], st),
        "psso_evaluate": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], st),
        "psso_evaluate_noalloc": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], st),
        "psso_fitness_forward": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p], st),
        "psso_fitness_backward": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], st),
        "psso_fitness_workspace_size": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_size_t)], st),
        "psso_fitness_forward_ws": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p], st),
        "psso_fitness_backward_ws": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p], st),
        "psso_rotate": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], st),
        "psso_time_kernels": ([H, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32], st),
        "psso_polish": ([H, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                         ctypes.POINTER(ctypes.c_int32)], st),
        "psso_autotune": ([ctypes.POINTER(psso_problem), ctypes.c_int32,
                           ctypes.POINTER(psso_config), ctypes.c_int32,
                           ctypes.POINTER(psso_config), ctypes.POINTER(psso_tune_report)], st),
        "psso_microbench": ([ctypes.POINTER(psso_peaks), ctypes.c_void_p], st),
        "psso_create_shard": ([ctypes.POINTER(psso_problem), ctypes.c_int64, ctypes.c_int64,
                               ctypes.POINTER(psso_config), ctypes.POINTER(H)], st),
        "psso_set_gbest": ([H, ctypes.c_int32, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p], st),
        "psso_check_report": ([ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                               ctypes.c_int32], st),
        "psso_check_selftest": ([ctypes.c_int64, ctypes.c_void_p], st),
        "psso_last_error": ([], ctypes.c_char_p),
        "psso_destroy": ([H], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status):
    if status != PSSO_OK:
        raise PssoError(status, load().psso_last_error().decode())


def _f64(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


# --- the C ABI, one function each ------------------------------------------------
def psso_create(fn, N, D, lb, ub, Cg, Cp, Cw, seed):
    h = ctypes.c_void_p()
    _check(load().psso_create(int(fn), N, D, lb, ub, Cg, Cp, Cw, seed, ctypes.byref(h)))
    return h


_CONFIG_KEYS = ("threads_per_block", "single_block_max", "log_stride", "log_capacity",
                "spin_limit", "stream", "max_blocks", "fault_skip_rank", "residency", "pipeline",
                "tensor_rotation", "batch_stream", "batch_blocks_per_sm", "flow")
FLOW = {"sync": PSSO_FLOW_SYNC, "async": PSSO_FLOW_ASYNC}


def _config(precision, opts):
    if isinstance(precision, str):
        precision = PRECISION[precision]
    bad = set(opts) - set(_CONFIG_KEYS)
    if bad:
        raise TypeError(f"unknown configuration fields {sorted(bad)}")
    cfg = psso_config()
    cfg.precision = int(precision)
    for k, v in opts.items():
        if k == "flow" and isinstance(v, str):
            v = FLOW[v]
        setattr(cfg, k, v)
    return cfg


def _problems(problems):
    arr = (psso_problem * len(problems))()
    keep = []
    for k, p in enumerate(problems):
        D = int(p["D"])
        o = _f64(p.get("o", p.get("shift")), D)
        w = _f64(p.get("w", p.get("weights")), D)
        M = _f64(p.get("M", p.get("rotation")), D * D)
        keep += [o, w, M]
        fn = p["fn"]
        lat = p.get("lattice", PSSO_LATTICE_F64)
        order = p.get("order", PSSO_ORDER_GPX)
        arr[k] = psso_problem(FN[fn] if isinstance(fn, str) else int(fn),
                              LATTICE[lat] if isinstance(lat, str) else int(lat),
                              int(p["N"]), D, float(p["lb"]), float(p["ub"]), float(p["Cg"]),
                              float(p["Cp"]), float(p["Cw"]), int(p["seed"]),
                              int(p.get("sid", p.get("stream_id", 0))),
                              ORDER[order] if isinstance(order, str) else int(order),
                              _ptr(o), _ptr(w), _ptr(M))
    return arr, keep


def psso_create_ex(problems, precision=PSSO_PREC_F64, **config):
    """``problems``: list of dicts with keys fn, N, D, lb, ub, Cg, Cp, Cw, seed and
    optional lattice, sid / stream_id, order ("gpx" / "paper"), o / shift,
    w / weights, M / rotation.
    ``config``: any psso_config field by name (threads_per_block, log_stride,
    log_capacity, stream, batch_blocks_per_sm, ...)."""
    arr, keep = _problems(problems)
    cfg = _config(precision, config)
    h = ctypes.c_void_p()
    _check(load().psso_create_ex(arr, len(problems), ctypes.byref(cfg), ctypes.byref(h)))
    return h


def psso_create_shard(problem, first, count, precision=PSSO_PREC_F64, **config):
    """Handle for particles first .. first+count-1 of one swarm (see psso.h)."""
    arr, keep = _problems([problem])
    cfg = _config(precision, config)
    h = ctypes.c_void_p()
    _check(load().psso_create_shard(arr, int(first), int(count), ctypes.byref(cfg),
                                    ctypes.byref(h)))
    return h


def psso_set_gbest(h, instance, value, index, row):
    """Replace the gBest the next generation searches with (value, index, row)."""
    row = np.ascontiguousarray(row, dtype=np.float64)
    _check(load().psso_set_gbest(h, int(instance), float(value), int(index), _ptr(row)))


def psso_autotune(problems, precision=PSSO_PREC_F64, generations=200, **config):
    """Launch-shape autotuner: returns (fields, report) where ``fields`` is a
    dict of the tuned psso_config fields (threads_per_block,
    batch_blocks_per_sm) to pass on to psso_create_ex, and ``report`` a dict
    (candidates, best_ms, default_ms per generation)."""
    arr, keep = _problems(problems)
    cfg = _config(precision, config)
    out = psso_config()
    rep = psso_tune_report()
    _check(load().psso_autotune(arr, len(problems), ctypes.byref(cfg), int(generations),
                                ctypes.byref(out), ctypes.byref(rep)))
    fields = {"threads_per_block": out.threads_per_block,
              "batch_blocks_per_sm": out.batch_blocks_per_sm}
    report = {"candidates": rep.candidates, "threads_per_block": rep.threads_per_block,
              "batch_blocks_per_sm": rep.batch_blocks_per_sm, "best_ms": rep.best_ms,
              "default_ms": rep.default_ms}
    return fields, report


def psso_run(h, generations):
    _check(load().psso_run(h, int(generations)))


def psso_reset(h):
    _check(load().psso_reset(h))


def psso_sync(h):
    _check(load().psso_sync(h))


def psso_best(h, instance=0, D=None):
    """Returns (value, index, row); row has D values when D is given."""
    v = ctypes.c_double()
    i = ctypes.c_int64()
    row = None if D is None else np.empty(int(D), dtype=np.float64)
    _check(load().psso_best(h, instance, ctypes.byref(v), ctypes.byref(i), _ptr(row)))
    return v.value, i.value, row


def psso_get_state(h, instance, N, D):
    X = np.empty((N, D), dtype=np.float64)
    P = np.empty((N, D), dtype=np.float64)
    pF = np.empty(N, dtype=np.float64)
    _check(load().psso_get_state(h, instance, _ptr(X), _ptr(P), _ptr(pF)))
    return X, P, pF


def psso_get_log(h, instance=0, cap=1 << 20):
    n = ctypes.c_int64()
    _check(load().psso_get_log(h, instance, None, 0, ctypes.byref(n)))
    m = min(cap, n.value)
    buf = (psso_log_entry * max(1, m))()
    _check(load().psso_get_log(h, instance, ctypes.addressof(buf), m, ctypes.byref(n)))
    out = {k: np.empty(n.value, dtype=dt) for k, dt in
           (("generation", np.int64), ("index", np.int64), ("value", np.float64),
            ("value_lo", np.float32), ("value_hi", np.float32), ("accepted", np.int64),
            ("rechecks", np.int64))}
    for q in range(n.value):
        for k in out:
            out[k][q] = getattr(buf[q], k)
    return out


def psso_stats(h):
    s = psso_stats_t()
    _check(load().psso_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in psso_stats_t._fields_ if k != "reserved"}


def psso_generation(h):
    return int(load().psso_generation(h))


def psso_save(h):
    n = ctypes.c_size_t()
    _check(load().psso_save(h, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().psso_save(h, buf, n.value, ctypes.byref(n)))
    return buf.raw


def psso_load(h, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    _check(load().psso_load(h, buf, len(data)))


def psso_evaluate(fn, X, shift=None, weights=None, rotation=None, precision=PSSO_PREC_F64,
                  stream=None):
    """Batched fitness of the rows of X (N x D).  Returns (f, err)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[None, :]
    N, D = X.shape
    o = _f64(shift, D)
    w = _f64(weights, D)
    M = _f64(rotation, D * D)
    if isinstance(fn, str):
        fn = FN[fn]
    if isinstance(precision, str):
        precision = PRECISION[precision]
    f = np.empty(N, dtype=np.float64)
    e = np.empty(N, dtype=np.float64)
    _check(load().psso_evaluate(int(fn), N, D, _ptr(X), _ptr(o), _ptr(w), _ptr(M),
                                int(precision), _ptr(f), _ptr(e), stream))
    return f, e


def psso_evaluate_noalloc(fn, N, D, X_ptr, shift_ptr, weights_ptr, precision, f_ptr, err_ptr,
                          stream=None):
    """Allocation-free batched fitness on device buffers (raw device pointers,
    e.g. ``tensor.data_ptr()``).  Enqueued on ``stream``; does not wait."""
    if isinstance(fn, str):
        fn = FN[fn]
    if isinstance(precision, str):
        precision = PRECISION[precision]
    _check(load().psso_evaluate_noalloc(int(fn), int(N), int(D), X_ptr, shift_ptr, weights_ptr,
                                        int(precision), f_ptr, err_ptr, stream))


def psso_fitness_forward(fn, N, D, X_ptr, shift_ptr, weights_ptr, rotation_ptr, f_ptr,
                         stream=None):
    """FP32 batched fitness on device buffers (raw float32 device pointers).
    Enqueued on ``stream``; does not wait."""
    if isinstance(fn, str):
        fn = FN[fn]
    _check(load().psso_fitness_forward(int(fn), int(N), int(D), X_ptr, shift_ptr, weights_ptr,
                                       rotation_ptr, f_ptr, stream))


def psso_fitness_backward(fn, N, D, X_ptr, shift_ptr, weights_ptr, rotation_ptr, grad_f_ptr,
                          grad_X_ptr, stream=None):
    """grad_X = grad_f[:, None] * df/dX on device buffers (raw float32 device
    pointers).  Enqueued on ``stream``; does not wait."""
    if isinstance(fn, str):
        fn = FN[fn]
    _check(load().psso_fitness_backward(int(fn), int(N), int(D), X_ptr, shift_ptr, weights_ptr,
                                        rotation_ptr, grad_f_ptr, grad_X_ptr, stream))


def psso_fitness_workspace_size(fn, N, D):
    """Device bytes the tensor-core fitness calls need (0: none)."""
    if isinstance(fn, str):
        fn = FN[fn]
    n = ctypes.c_size_t(0)
    _check(load().psso_fitness_workspace_size(int(fn), int(N), int(D), ctypes.byref(n)))
    return int(n.value)


def psso_fitness_forward_ws(fn, N, D, X_ptr, shift_ptr, weights_ptr, rotation_ptr, f_ptr,
                            ws_ptr, ws_bytes, stream=None):
    """psso_fitness_forward with the rotated product on the tensor cores
    (caller-owned device workspace).  Does not wait."""
    if isinstance(fn, str):
        fn = FN[fn]
    _check(load().psso_fitness_forward_ws(int(fn), int(N), int(D), X_ptr, shift_ptr, weights_ptr,
                                          rotation_ptr, f_ptr, ws_ptr, int(ws_bytes), stream))


def psso_fitness_backward_ws(fn, N, D, X_ptr, shift_ptr, weights_ptr, rotation_ptr, grad_f_ptr,
                             grad_X_ptr, ws_ptr, ws_bytes, stream=None):
    """psso_fitness_backward with both rotated products on the tensor cores
    (caller-owned device workspace).  Does not wait."""
    if isinstance(fn, str):
        fn = FN[fn]
    _check(load().psso_fitness_backward_ws(int(fn), int(N), int(D), X_ptr, shift_ptr, weights_ptr,
                                           rotation_ptr, grad_f_ptr, grad_X_ptr, ws_ptr,
                                           int(ws_bytes), stream))


def psso_rotate(N, D, X_ptr, shift_ptr, rotation_ptr, Z_ptr, stream=None):
    """Z = (X - o) M^T on the tensor cores (raw float32 device pointers).
    Synchronises ``stream``."""
    _check(load().psso_rotate(int(N), int(D), X_ptr, shift_ptr, rotation_ptr, Z_ptr, stream))


PIPELINE_KERNELS = ("update", "gemm_fit", "decide", "z32", "fix32", "z64", "fix64", "argmin0",
                    "z64_argmin", "fix64_argmin", "argmin1")


def psso_time_kernels(h, instance=0, generations=10):
    """Mean duration (ms) of each kernel of a tensor-pipeline generation."""
    ms = (ctypes.c_float * 16)()
    _check(load().psso_time_kernels(h, int(instance), int(generations), ctypes.addressof(ms), 16))
    return dict(zip(PIPELINE_KERNELS, list(ms)[:len(PIPELINE_KERNELS)]))


BATCH_KERNELS = ("stream", "step", "argmin")


def psso_time_batch_kernels(h, generations=10):
    """psso_time_kernels on a handle that runs the batched pipeline: mean ms
    per generation of its streaming step kernels, other step kernels and
    arg-min kernel."""
    ms = (ctypes.c_float * 16)()
    _check(load().psso_time_kernels(h, 0, int(generations), ctypes.addressof(ms), 16))
    return dict(zip(BATCH_KERNELS, list(ms)[:3]))


def psso_polish(h, instance=0, steps=20, lr=1e-3):
    """Gradient polish of the gBest row of ``instance``; returns True when it
    replaced the gBest particle's pBest (strictly lower FP64 fitness)."""
    improved = ctypes.c_int32(0)
    _check(load().psso_polish(h, int(instance), int(steps), float(lr), ctypes.byref(improved)))
    return bool(improved.value)


def psso_microbench(stream=None):
    """Measured peaks of the current GPU (dict of psso_peaks fields)."""
    out = psso_peaks()
    _check(load().psso_microbench(ctypes.byref(out), stream))
    return {k: getattr(out, k) for k, _ in psso_peaks._fields_ if k != "reserved"}


CHECK_SITES = {1: "selftest", 2: "unit range", 3: "unit shared memory", 4: "row", 5: "exchange slot",
               6: "log entry", 7: "gBest source row", 8: "refined row", 9: "batched instance",
               10: "batched row", 11: "list slot", 12: "tensor-pipeline row", 13: "evaluated row",
               14: "asynchronous-flow row", 15: "GEMM tile"}


def psso_check_report(clear=False):
    """First failed index check of a checked build: (site, index), site 0 if none."""
    site, index = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(load().psso_check_report(ctypes.byref(site), ctypes.byref(index), 1 if clear else 0))
    return site.value, index.value


def psso_check_selftest(index, stream=None):
    _check(load().psso_check_selftest(int(index), stream))


def psso_last_error():
    return load().psso_last_error().decode()


def psso_destroy(h):
    if h is not None and h.value:
        load().psso_destroy(h)
        h.value = None
