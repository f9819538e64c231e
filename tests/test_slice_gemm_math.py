"""The arithmetic of the tensor pipeline's exact integer-slice GEMM, restated
in numpy float32 on the CPU: the slice scale, the four 6-bit slices and the
facts the bound rests on -- |V0| <= 63, |V1..V3| <= 32, the remainder below
2^-25, every accumulator's partial sums below 2^23 for K <= 1024, and the
dropped slice products within SLICE_DROP per k."""
import numpy as np

F = np.float32
SLICE_DROP = 3.04 * 2.0 ** -26 + 3 * 2.0 ** -50


def slice_scale(vmax):
    if not vmax > 0:
        return F(1.0)
    m = F(F(F(vmax) * F(64.0 / 63.0)) * F(1 + 2.0 ** -20))
    _, e = np.frexp(m)
    return F(np.ldexp(1.0, int(e)))


def slice4(u):
    """Slices of float32 u (|u| <= 63/64), each step in float32."""
    w = F(u) * F(64.0)
    out = []
    for _ in range(4):
        q = np.rint(w).astype(F)
        out.append(q)
        w = F(F(w - q) * F(64.0))
    return np.array(out, dtype=np.float64)


def _rows(rng, n, D):
    scale = 10.0 ** rng.uniform(-6, 3, (n, 1))
    v = (rng.standard_normal((n, D)) * scale).astype(F)
    v[0, :] = 0
    v[1, :D // 2] = F(2.0 ** -140)          # subnormal-range values next to normal ones
    return v


def test_slices_reconstruct_within_remainder_bound():
    rng = np.random.default_rng(7)
    for row in _rows(rng, 60, 257):
        s = slice_scale(float(np.abs(row).max()))
        assert np.abs(row).max() <= 63 / 64 * s
        for v in row:
            u = F(v) * F(1.0 / s)
            sl = slice4(u)
            assert abs(sl[0]) <= 63 and np.all(np.abs(sl[1:]) <= 32)
            assert np.all(sl == np.rint(sl))
            rec = sum(sl[q] * 64.0 ** -(q + 1) for q in range(4))
            assert abs(float(u) - rec) <= 2.0 ** -25


def test_edge_values():
    for u in (63 / 64, -63 / 64, 0.5, 2.0 ** -24, 2.0 ** -25, 2.0 ** -26, 1 / 128 - 2.0 ** -30):
        sl = slice4(F(u))
        rec = sum(sl[q] * 64.0 ** -(q + 1) for q in range(4))
        assert abs(float(F(u)) - rec) <= 2.0 ** -25
        assert abs(sl[0]) <= 63 and np.all(np.abs(sl[1:]) <= 32)


def test_accumulators_exact_and_dropped_terms_bounded():
    """Per k the weight-w slice products sum to at most 3969 / 4032 / 5056 /
    6080, so K = 1024 partial sums stay below 2^23; the products of weight
    4..6 and the remainders are within the per-k bound the epilogue uses."""
    rng = np.random.default_rng(11)
    D = 1000
    d = _rows(rng, 6, D)
    M = _rows(rng, 6, D)
    for dr in d:
        sd = slice_scale(float(np.abs(dr).max()))
        Sd = np.array([slice4(F(v) * F(1.0 / sd)) for v in dr])          # [D][4]
        for mr in M:
            sm = slice_scale(float(np.abs(mr).max()))
            Sm = np.array([slice4(F(v) * F(1.0 / sm)) for v in mr])
            kept = np.zeros(D)
            for w in range(4):
                prod = sum(Sd[:, q] * Sm[:, w - q] for q in range(w + 1))
                assert np.abs(prod).max() <= (3969, 4032, 5056, 6080)[w]
                assert np.abs(prod).sum() < 2 ** 23
                kept += prod * 64.0 ** -(w + 2)
            exact = dr.astype(np.float64) * mr.astype(np.float64)
            dropped = np.abs(exact - kept * float(sd) * float(sm))
            bound = SLICE_DROP * float(sd) * float(sm) + 2.0 ** -25 * (
                float(sm) * np.abs(dr.astype(np.float64)) + float(sd) * np.abs(mr.astype(np.float64)))
            assert np.all(dropped <= bound * (1 + 1e-12))
