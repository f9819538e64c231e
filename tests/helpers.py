"""Shared checks of the GPU tests (no GPU needed to import)."""
import numpy as np

# The precision form's target: FP32 fitness within 1e-6 relative of the FP64
# value; Ackley's optimum is 0, so its error is taken relative to
# max(|f|, 1e-6 (20 + e)).
REL_TOL = 1e-6


def fitness_rel_err(f_gpu, f_ref, fn):
    """Element-wise |f_gpu - f_ref| / max(|f_ref|, floor(fn))."""
    f_gpu = np.asarray(f_gpu, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    floor = 1e-6 * (20 + np.e) if fn.endswith("ackley") else 0.0
    scale = np.maximum(np.abs(f_ref), floor)
    return np.abs(f_gpu - f_ref) / np.where(scale > 0, scale, 1.0)
