"""The arithmetic of the tensor pipeline's exact integer-slice GEMM, restated
in numpy on the CPU: the slice scale, the four 7-bit slices of an exact float
pair (d = x - o) and of an FP64 value (M), and the facts the bound rests on --
|V0..V3| <= 64, the rest within 1.01 2^-29, the four accumulators (one per
weight) gaining per k at most 4096 / 8192 / 12288 / 16384 so that partial sums
over D <= 1023 terms stay below 2^24, and the dropped products of weight 4..6
with the remainders within the per-k bound of the epilogue."""
import numpy as np

F = np.float32
SLICE_DROP = 3.04 * 2.0 ** -30
SLICE_REM = 1.01 * 2.0 ** -29
# (A slice, B slice) pairs of each accumulator, its weight, its per-k maximum
ACCS = [([(0, 0)], 0, 4096), ([(0, 1), (1, 0)], 1, 8192), ([(0, 2), (1, 1), (2, 0)], 2, 12288),
        ([(0, 3), (1, 2), (2, 1), (3, 0)], 3, 16384)]


def slice_scale(vmax):
    if not vmax > 0:
        return F(1.0)
    m = F(F(F(vmax) * F(2.0)) * F(1 + 2.0 ** -20))
    _, e = np.frexp(m)
    return F(np.ldexp(1.0, int(e)))


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def slice_pair(hi, lo):
    """Slices of the float32 pair hi + lo, every step in float32."""
    wh, wl = F(hi * F(128)), F(lo * F(128))
    out = []
    for _ in range(4):
        q = F(np.rint(wh))
        out.append(float(q))
        r = F(wh - q)
        s, e = two_sum(r, wl)
        wh, wl = F(s * F(128)), F(e * F(128))
    return np.array(out)


def slice_f64(u):
    w = u * 128.0
    out = []
    for _ in range(4):
        q = np.rint(w)
        out.append(q)
        w = (w - q) * 128.0
    return np.array(out)


def _d_rows(rng, n, D):
    """d = x - o for float32 x and o, as exact float pairs (and in float64)."""
    rows = []
    for t in range(n):
        scale = 10.0 ** rng.uniform(-3, 3)
        x = (rng.uniform(-1, 1, D) * scale).astype(F)
        o = (rng.uniform(-1, 1, D) * scale * rng.uniform(0, 2)).astype(F)
        if t == 0:
            x = o.copy()                                 # d = 0
        pairs = [two_sum(a, F(-b)) for a, b in zip(x, o)]
        hi = np.array([p[0] for p in pairs], F)
        lo = np.array([p[1] for p in pairs], F)
        exact = x.astype(np.float64) - o.astype(np.float64)
        assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), exact)
        rows.append((hi, lo, exact))
    return rows


def _d_slices(hi, lo):
    l1 = float(F(np.abs(hi).sum(dtype=np.float64) * (1 + 2.0 ** -22)))
    sd = slice_scale(float(np.abs(hi).max()))
    inv = F(1.0 / sd)
    S = np.array([slice_pair(F(h * inv), F(l * inv)) for h, l in zip(hi, lo)])
    return float(sd), S, l1


def _m_slices(m):
    sm = slice_scale(float(F(np.abs(m).max()) * F(1 + 2.0 ** -23)))
    return float(sm), np.array([slice_f64(v / float(sm)) for v in m])


def test_slices_reconstruct_within_remainder_bound():
    rng = np.random.default_rng(7)
    for hi, lo, exact in _d_rows(rng, 20, 129):
        sd, S, _ = _d_slices(hi, lo)
        assert np.abs(exact).max() < sd / 2
        assert np.all(np.abs(S) <= 64)
        rec = S @ (128.0 ** -np.arange(1, 5))
        assert np.all(np.abs(exact / sd - rec) <= SLICE_REM)
    for _ in range(20):
        m = rng.standard_normal(129) * 10.0 ** rng.uniform(-4, 1)
        sm, S = _m_slices(m)
        assert np.abs(m).max() < sm / 2
        assert np.all(np.abs(S) <= 64)
        assert np.all(np.abs(m / sm - S @ (128.0 ** -np.arange(1, 5))) <= SLICE_REM)


def test_accumulators_exact_and_dropped_terms_bounded():
    rng = np.random.default_rng(11)
    D = 1000
    for hi, lo, exact in _d_rows(rng, 4, D):
        sd, Sd, l1d = _d_slices(hi, lo)
        assert np.abs(exact).sum() <= l1d
        for _ in range(4):
            m = rng.standard_normal(D) * 10.0 ** rng.uniform(-3, 0)
            sm, Sm = _m_slices(m)
            kept = np.zeros(D)
            for pairs, w, cap in ACCS:
                prod = sum(Sd[:, a] * Sm[:, b] for a, b in pairs)
                assert np.abs(prod).max() <= cap
                assert np.abs(prod).sum() < 2 ** 24
                kept += prod * 128.0 ** -(w + 2)
            dropped = np.abs(exact * m - kept * sd * sm)
            bound = SLICE_DROP * sd * sm + SLICE_REM * (sm * np.abs(exact) + sd * np.abs(m))
            assert np.all(dropped <= bound * (1 + 1e-9))


def test_extreme_slices_and_worst_case_partial_sums():
    """Entries at the row maximum give a top slice of magnitude 64, never
    more; with every slice at 64 the per-k gains of the four accumulators are
    1, 2, 3 and 4 products of 4096, and over D <= 1023 terms the partial sums
    stay below 2^24 (with D = 1024 the last could reach it, hence the limit)."""
    m = np.array([1.99, -1.99, 1.9921875, 0.25, -1e-9, 0.0])
    sm, S = _m_slices(m)
    assert sm == 4.0 and np.abs(m).max() < sm / 2 and np.all(np.abs(S) <= 64)
    assert np.abs(S[:, 0]).max() == 64
    for pairs, _, cap in ACCS:
        assert cap == 4096 * len(pairs)
        assert cap * 1023 < 2 ** 24
    assert max(cap for _, _, cap in ACCS) * 1024 == 2 ** 24
