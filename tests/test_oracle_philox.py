"""Pins for the oracle's Philox-4x32-10 and its fresh-value lattices.

The reference is Triton's own Philox-4x32-10 (``tl.philox``), run on the CPU by
Triton's interpreter in a child process: an implementation written by other
people from the same published definition (Salmon et al., SC'11)."""
import json
from fractions import Fraction
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r'''
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(out, c0p, c1p, c2p, c3p, seed, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c0p + offs); c1 = tl.load(c1p + offs)
    c2 = tl.load(c2p + offs); c3 = tl.load(c3p + offs)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out + offs * 4 + 0, a); tl.store(out + offs * 4 + 1, b)
    tl.store(out + offs * 4 + 2, c); tl.store(out + offs * 4 + 3, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    ctrs = np.array(ctrs, dtype=np.uint32).reshape(-1, 4)
    m = ctrs.shape[0]
    n = 1 << max(0, (m - 1).bit_length())          # tl.arange needs a power of two
    ctrs = np.concatenate([ctrs, np.zeros((n - m, 4), dtype=np.uint32)])
    cols = [torch.from_numpy(np.ascontiguousarray(ctrs[:, q]).view(np.int32)).view(torch.uint32)
            for q in range(4)]
    out = torch.zeros(4 * n, dtype=torch.uint32)
    k[(1,)](out, *cols, seed, n=n)
    res.append(out.view(torch.int32).numpy().view(np.uint32).reshape(n, 4)[:m].tolist())
print(json.dumps(res))
'''


def _triton_philox(requests):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(requests),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr.strip().splitlines()[-1])
    return json.loads(p.stdout)


def _requests():
    rng = np.random.default_rng(7)
    reqs = []
    for seed in (0, 1, 0xFFFFFFFF, 0x123456789ABCDEF0, 2**64 - 1):
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = 2**32 - 1
        ctrs[2] = [5, 7, 3, (3 | (9 << 8))]        # (block, particle, generation, tag|stream)
        reqs.append([int(seed), ctrs.astype(np.uint32).tolist()])
    return reqs


def test_philox_matches_triton():
    reqs = _requests()
    ref = _triton_philox(reqs)
    for (seed, ctrs), outs in zip(reqs, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, expect in zip(ctrs, outs):
            got = oracle.philox(c, key)
            assert got.tolist() == expect, (seed, c)


def test_philox_round_is_a_bijection_on_counters():
    # Distinct counters under one key give distinct blocks (Philox is a keyed
    # bijection); a dropped or duplicated round constant usually breaks this
    # for structured counters.
    seen = set()
    for a in range(64):
        for b in range(64):
            seen.add(tuple(oracle.philox([a, b, 0, 0], [1, 0]).tolist()))
    assert len(seen) == 64 * 64


def test_philox_words_uniform():
    # Chi-square on the top 8 bits of 2^16 words from a counter sweep.
    words = np.concatenate([oracle.philox([c, 3, 1, 2], [1, 0]) for c in range(1 << 14)])
    hist = np.bincount((words >> 24).astype(np.int64), minlength=256)
    e = words.size / 256
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 255 + 6 * np.sqrt(2 * 255)


def test_fresh_lattice_maps_triton_words():
    """fresh() = the lattice map of the Philox words at its counter."""
    seed, sid, g = 1, 3, 7
    cases = [(i, j) for i in (0, 5, 1023) for j in (0, 1, 2, 3, 6, 99)]
    reqs = [[seed, [[j >> 1, i, g, oracle.TAG_FRESH | (sid << 8)] for i, j in cases]],
            [seed, [[j >> 2, i, g, oracle.TAG_FRESH | (sid << 8)] for i, j in cases]]]
    w64, w32 = _triton_philox(reqs)
    lb, ub = -5.12, 5.12
    for (i, j), a, b in zip(cases, w64, w32):
        m = ((a[2 * (j & 1) + 1] << 32) | a[2 * (j & 1)]) >> 11
        expect64 = min(max(np.fma(ub - lb, m / 2.0**53, lb) if hasattr(np, "fma") else
                           float(np.float64(ub - lb) * (m / 2.0**53) + lb), lb), ub)
        got64 = oracle.fresh("f64", seed, sid, oracle.TAG_FRESH, g, i, j, lb, ub)
        assert abs(got64 - expect64) <= 2 * np.spacing(ub)
        m32 = b[j & 3] >> 8
        S, L = np.float32(ub - lb), np.float32(lb)
        expect32 = _rn32(Fraction(float(S)) * Fraction(m32, 2**24) + Fraction(float(L)))
        expect32 = min(max(expect32, _float_ge(lb)), _float_le(ub))
        got32 = oracle.fresh("f32", seed, sid, oracle.TAG_FRESH, g, i, j, lb, ub)
        assert got32 == expect32
        assert lb <= got32 <= ub


def _rn32(fr):
    """Nearest float32 (ties to even) to the exact rational fr."""
    f = np.float32(float(fr))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - fr),
                                     int(np.array(c, dtype=np.float32).view(np.uint32)) & 1))
    return float(best)


def _float_ge(v):
    f = np.float32(v)
    return float(np.nextafter(f, np.float32(np.inf)) if float(f) < v else f)


def _float_le(v):
    f = np.float32(v)
    return float(np.nextafter(f, np.float32(-np.inf)) if float(f) > v else f)


def test_fresh_exact_unit_interval():
    # On [0, 1] the FP64 lattice value is u = m 2^-53 exactly.
    for i in range(4):
        for j in range(8):
            x = oracle.fresh("f64", 9, 0, oracle.TAG_INIT, 0, i, j, 0.0, 1.0)
            m = x * 2.0**53
            assert m == int(m) and 0 <= m < 2**53


@pytest.mark.parametrize("lattice", ["f64", "f32"])
def test_fresh_range_and_uniformity(lattice):
    lb, ub = -2.048, 2.048
    xs = np.array([oracle.fresh(lattice, 1, 0, oracle.TAG_FRESH, 1, i, j, lb, ub)
                   for i in range(128) for j in range(128)])
    assert xs.min() >= lb and xs.max() <= ub
    hist = np.histogram(xs, bins=64, range=(lb, ub))[0]
    e = xs.size / 64
    assert ((hist - e) ** 2 / e).sum() < 63 + 6 * np.sqrt(2 * 63)
    if lattice == "f32":
        assert np.all(xs.astype(np.float32).astype(np.float64) == xs)


def test_fresh_stays_inside_unrepresentable_bounds():
    # Bounds that are not floats: every FP32-lattice value must still lie in [lb, ub].
    lb, ub = -0.1, 0.30000000000000004
    for j in range(512):
        x = oracle.fresh("f32", 11, 0, oracle.TAG_FRESH, 2, 1, j, lb, ub)
        assert lb <= x <= ub
