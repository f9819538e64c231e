"""The accumulation model behind every tensor-core bound (tc_gemm.cuh
MMA_EPS): one kind::f16 MMA with FP32 accumulation adds its 16 exact
BF16 x BF16 products to the accumulator with an error of at most
MMA_EPS * (|accumulator| + sum |products|), MMA_EPS = 2^-20.

The probes go through psso_rotate with BF16-exact operands (the split's
second and third parts are zero, so each output is the first accumulator
chain alone) and every nonzero entry in the first 64-wide K block: output j
of row i is then the chain of four MMAs over k = 0..15, 16..31, 32..47,
48..63, the first without an accumulator.  Exact sums are integers (every
product is a multiple of 2^-53 below 2); the bound follows the chain step by
step.  The adversarial rows put addends just below the quarter-ulp grid of
the largest addend, where an aligning adder that truncates loses them whole."""
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MMA_EPS = Fraction(1, 2 ** 20)
D = 192                      # three K blocks; only the first holds products
SCALE = 2 ** 53


def _rotate(lib, X, M):
    N = X.shape[0]
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Md = torch.tensor(M, dtype=torch.float32, device="cuda")
    o = torch.zeros(D, dtype=torch.float32, device="cuda")
    Z = torch.full((N, D), float("nan"), dtype=torch.float32, device="cuda")
    lib.psso_rotate(N, D, Xd.data_ptr(), o.data_ptr(), Md.data_ptr(), Z.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return Z.cpu().numpy()


def _bf16_exact(a):
    b = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy()
    return np.array_equal(b, a)


def _check(lib, X, rows):
    """Returns (worst error / model bound, worst error / derived worst case)."""
    worst = worst_derived = 0.0
    for c in range(0, len(rows), D):              # M is D x D: D probe rows per call
        w, wd = _check_block(lib, X, np.stack(rows[c:c + D]))
        worst, worst_derived = max(worst, w), max(worst_derived, wd)
    return worst, worst_derived


def _check_block(lib, X, Mrows):
    M = np.zeros((D, D), np.float32)
    M[:len(Mrows)] = Mrows
    assert _bf16_exact(X) and _bf16_exact(M) and not np.any(M[:, 64:]) and not np.any(X[:, 64:])
    Z = _rotate(lib, X, M)
    # products as integers: every one is a multiple of 2^-53 of magnitude < 2
    Pi = np.rint(np.einsum("ik,jk->ijk", X[:, :64].astype(np.float64), M[:, :64].astype(np.float64))
                 * SCALE).astype(np.int64)
    worst = worst_derived = Fraction(0)
    for i in range(X.shape[0]):
        for j in range(len(Mrows)):
            row = Pi[i, j]
            acc = 0                 # exact partial sum (scaled)
            bound = Fraction(0)     # model bound on the accumulator's error so far
            derived = Fraction(0)   # the same with 0.625 * 2^-20
            for s in range(4):
                grp = row[16 * s:16 * s + 16]
                mag = ((abs(acc) + bound * SCALE) if s else 0) + int(np.abs(grp).sum())
                bound += MMA_EPS * Fraction(mag) / SCALE
                derived += Fraction(5, 8) * MMA_EPS * Fraction(mag) / SCALE
                acc += int(grp.sum())
            err = abs(Fraction(float(Z[i, j])) - Fraction(acc, SCALE))
            if err:
                assert err <= bound, (i, j, float(err), float(bound))
                worst = max(worst, err / bound)
                worst_derived = max(worst_derived, err / derived)
    return float(worst), float(worst_derived)


def _row(entries):
    r = np.zeros(D, np.float32)
    for k, v in entries:
        r[k] = np.float32(v)
    return r


def test_adversarial_rows_within_model(lib):
    rows = []
    for e in range(22, 33):
        for mant in (1.0, 1 - 2.0 ** -7, 1.5):
            t = mant * 2.0 ** -e
            for sg in (1.0, -1.0):
                rows.append(_row([(0, 1.0)] + [(k, sg * t) for k in range(1, 16)]))     # dominant first
                rows.append(_row([(15, 1.0)] + [(k, sg * t) for k in range(15)]))       # dominant last
                rows.append(_row([(0, 1.0)] + [(k, sg * t) for k in range(16, 64)]))    # large accumulator
                rows.append(_row([(k, sg * t) for k in range(48)] + [(48, 1.0)]))       # small accumulator
            rows.append(_row([(0, 1.0), (1, -(1 - 2.0 ** -8))] + [(k, t) for k in range(2, 16)]))
    X = np.ones((1, D), np.float32)
    X[:, 64:] = 0
    worst, worst_derived = _check(lib, X, rows)
    print(f"adversarial rows: worst error / bound {worst:.3f}, / derived worst case {worst_derived:.3f}")


def test_random_adversarial_rows_within_model(lib):
    rng = np.random.default_rng(2024)
    J, N = 96, 24
    M = np.zeros((J, D), np.float32)
    for j in range(J):
        base = rng.integers(0, 4)                     # exponent of the group's dominant term
        for k in range(64):
            # 8-bit significands, exponents clustered just below the quarter-ulp grid
            e = -int(base) - int(rng.choice([0, 1, 22, 23, 24, 25, 26, 27, 30, 40]))
            m = (128 + int(rng.integers(0, 128))) / 128.0
            M[j, k] = np.float32(rng.choice([-1.0, 1.0]) * m * 2.0 ** e)
    X = np.zeros((N, D), np.float32)
    X[:, :64] = (rng.choice([-1.0, 1.0], (N, 64)) * 2.0 ** rng.integers(-3, 1, (N, 64))).astype(np.float32)
    worst, worst_derived = _check(lib, X, list(M))
    print(f"random adversarial rows: worst error / bound {worst:.3f}, / derived worst case {worst_derived:.3f}")
