"""Tensor-core rotation z = M (x - o) (split BF16, tcgen05) against FP64.

The reference takes the same FP32 inputs d = fl32(x - o) and M32 = fl32(M)
and forms M32 d in FP64 (error ~1e-16 relative, negligible); the GPU result
must lie within the documented bound c(Kp) * sum_k |M32_jk| |d_k| +
2^-24 |z|, and the full error against the FP64 rotation of the exact
difference within the bound that includes the two input roundings."""
import numpy as np
import pytest
import torch

import workload

pytestmark = pytest.mark.gpu


def c_of(Kp):
    nkb = Kp // 64
    n0, n1 = 4 * ((nkb + 2) // 3), 5 * (Kp // 16)
    return 1.05 * (2.0 ** -20 * 1.04 * (n0 + n1 * 2.0 ** -7) + 1.03 * 2.0 ** -23 + 2.02 * 2.0 ** -24
                   + 3.1 * 2.0 ** -24)


def _rotate(lib, X32, o32, M32):
    N, D = X32.shape
    X = torch.tensor(X32, device="cuda")
    o = torch.tensor(o32, device="cuda")
    M = torch.tensor(M32, device="cuda")
    Z = torch.full((N, D), float("nan"), device="cuda")
    lib.psso_rotate(N, D, X.data_ptr(), o.data_ptr(), M.data_ptr(), Z.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    return Z.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,D", [(1, 1), (130, 37), (257, 64), (128, 100), (300, 256),
                                 (129, 1000), (64, 1025)])
def test_rotate_within_bound(lib, N, D):
    rng = np.random.default_rng(N * 7919 + D)
    M = workload.rotation(D, seed=3, stream=D % 5)
    M32 = M.astype(np.float32)
    o32 = rng.uniform(-80, 80, D).astype(np.float32)
    X32 = rng.uniform(-100, 100, (N, D)).astype(np.float32)
    Z = _rotate(lib, X32, o32, M32)
    d32 = (X32 - o32).astype(np.float32).astype(np.float64)
    Mf = M32.astype(np.float64)
    ref = d32 @ Mf.T
    S = np.abs(d32) @ np.abs(Mf).T
    Kp = (D + 63) // 64 * 64
    err = np.abs(Z - ref)
    bound = c_of(Kp) * S + 2.0 ** -24 * np.abs(Z)
    assert np.all(np.isfinite(Z))
    assert np.all(err <= bound), float((err / bound).max())
    # the model's slack: print the worst ratio for the record
    print(f"N={N} D={D}: max err / bound = {(err / np.maximum(bound, 1e-300)).max():.3e}, "
          f"max err / S = {(err / np.maximum(S, 1e-300)).max():.3e}")
    # against the FP64 rotation of the exact difference
    full = (X32.astype(np.float64) - o32.astype(np.float64)) @ M.T
    assert np.all(np.abs(Z - full) <= bound + 1.02 * 2.0 ** -23 * S)


def test_rotate_at_shift_is_zero(lib):
    D = 200
    M32 = workload.rotation(D, seed=4, stream=1).astype(np.float32)
    o32 = np.linspace(-3, 3, D).astype(np.float32)
    Z = _rotate(lib, np.tile(o32, (5, 1)), o32, M32)
    assert np.all(Z == 0.0)


def test_rotate_identity_is_exact(lib):
    """M = I: every product is d * 1 split exactly, so z = d bit for bit."""
    D, N = 96, 140
    rng = np.random.default_rng(5)
    X32 = rng.uniform(-5, 5, (N, D)).astype(np.float32)
    o32 = rng.uniform(-1, 1, D).astype(np.float32)
    Z = _rotate(lib, X32, o32, np.eye(D, dtype=np.float32))
    assert np.array_equal(Z, (X32 - o32).astype(np.float64))


def test_rotate_arguments_rejected(lib):
    with pytest.raises(lib.PssoError):
        lib.psso_rotate(0, 4, 1, 1, 1, 1)
    with pytest.raises(lib.PssoError):
        lib.psso_rotate(4, 0, 1, 1, 1, 1)
    with pytest.raises(lib.PssoError):
        lib.psso_rotate(4, 4, None, 1, 1, 1)
