"""Pins for the rest of Table 3.2 in the oracle: f2 hyper-ellipsoid, f3
Schwefel's problem 1.2, f7 Griewank, f8 Powell, f9 Schwefel.

Exact values at hand-computed points (integer arithmetic, where FP64 is exact),
the optimum at x = o, special cases that reduce to another function, an
mpmath evaluation of each textbook definition at random points (cos and sin
of the definition, not the sin(pi q) route the oracle takes), and, for f3, a
check that the blocked prefix-sum order stays within the FP64 error bound of
the exact prefix sums."""
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
import workload

mpmath.mp.prec = 200
EPS = 2.0**-53
NEW = ["hyper_ellipsoid", "schwefel12", "griewank", "powell", "schwefel"]


def _o(D, lo=-3.0, hi=3.0, seed=5):
    return workload.shift(D, lo, hi, seed)


def _f(fn, x, o):
    return oracle.fitness(fn, x, o)


@pytest.mark.parametrize("D", [1, 2, 5, 31, 100, 257, 1000])
def test_optimum_at_shift(D):
    o = _o(D)
    for fn in ["hyper_ellipsoid", "schwefel12", "griewank", "powell"]:
        assert _f(fn, o, o) == 0.0, fn
    # Schwefel at z = 0: every term z sin(sqrt|z|) is 0
    assert _f("schwefel", o, o) == 418.9829 * D


@pytest.mark.parametrize("D", [1, 4, 7, 64, 300])
def test_hyper_ellipsoid_exact(D):
    """Integer z: every operation is exact in FP64; at o + 1 the value is
    D (D + 1) / 2, and it equals the weighted ellipsoid with w_j = j + 1."""
    o = np.zeros(D)
    assert _f("hyper_ellipsoid", np.ones(D), o) == D * (D + 1) / 2
    ks = (np.arange(D) % 7 - 3).astype(np.float64)
    want = float(sum((j + 1) * int(k) ** 2 for j, k in enumerate(ks)))
    assert _f("hyper_ellipsoid", ks, o) == want
    x = np.random.default_rng(D).uniform(-5, 5, D)
    w = np.arange(1, D + 1, dtype=np.float64)
    assert _f("hyper_ellipsoid", x, o) == oracle.fitness("ellipsoid", x, o, w)


@pytest.mark.parametrize("D", [1, 3, 8, 129, 300, 1000])
def test_schwefel12_exact(D):
    """Integer z: prefix sums and squares are exact.  z = 1: c_j = j + 1, so
    f = D (D + 1)(2D + 1) / 6; a unit step at k: c_j = [j >= k], f = D - k."""
    o = np.zeros(D)
    assert _f("schwefel12", np.ones(D), o) == D * (D + 1) * (2 * D + 1) / 6
    for k in {0, D // 3, D - 1}:
        e = np.zeros(D)
        e[k] = 1.0
        assert _f("schwefel12", e, o) == D - k
    ks = (np.arange(D) % 5 - 2).astype(np.float64)
    c = np.cumsum(ks)
    assert _f("schwefel12", ks, o) == float((c * c).sum())


@pytest.mark.parametrize("D", [5, 130, 1000])
def test_schwefel12_against_exact_prefix(D):
    """Random z: the blocked prefix order of the oracle stays within the FP64
    bound of the exact value (every c_j has at most 4 + 5 + ceil(D/128) + 4
    roundings, each of at most EPS times a partial sum bounded by sum |z|)."""
    rng = np.random.default_rng(D)
    o = _o(D, seed=D)
    x = rng.uniform(-65, 65, D)
    z = [Fraction(float(a)) - Fraction(float(b)) for a, b in zip(x, o)]
    zf = (x - o)
    c, acc = [], Fraction(0)
    for zi in z:
        acc += zi
        c.append(acc)
    exact = float(sum(ci * ci for ci in c))
    A = float(np.abs(zf).sum())
    depth = 4 + 5 + -(-D // 128) + 4
    ec = 1.01 * (depth + 1) * EPS * A          # error of every c_j (z rounded once too)
    bound = sum(2 * abs(float(ci)) * ec + ec * ec for ci in c) + 2 * (D + 5) * EPS * exact
    assert abs(_f("schwefel12", x, o) - exact) <= bound


def _mp_griewank(z):
    s = mpmath.fsum(mpmath.mpf(float(v)) ** 2 for v in z) / 4000
    p = mpmath.fprod(mpmath.cos(mpmath.mpf(float(v)) / mpmath.sqrt(j + 1)) for j, v in enumerate(z))
    return 1 + s - p


def _mp_schwefel(z):
    return 418.9829 * len(z) - mpmath.fsum(
        mpmath.mpf(float(v)) * mpmath.sin(mpmath.sqrt(abs(mpmath.mpf(float(v))))) for v in z)


def _mp_powell(z):
    z = list(map(float, z)) + [0.0] * (-len(z) % 4)
    t = mpmath.mpf(0)
    for g in range(0, len(z), 4):
        a, b, c, d = (mpmath.mpf(v) for v in z[g:g + 4])
        t += (a + 10 * b) ** 2 + 5 * (c - d) ** 2 + (b - 2 * c) ** 4 + 10 * (a - d) ** 4
    return t


@pytest.mark.parametrize("D", [1, 2, 7, 50, 333])
def test_textbook_definitions_mpmath(D):
    """The oracle against mpmath evaluations of the textbook definitions (cos,
    sin, sqrt at 200 bits), with z = x - o formed exactly as the oracle does."""
    rng = np.random.default_rng(100 + D)
    for fn, (lb, ub) in (("griewank", (-600, 600)), ("schwefel", (-500, 500)), ("powell", (-4, 5))):
        o = workload.shift(D, 0.8 * lb, 0.8 * ub, 3)
        for x in rng.uniform(lb, ub, (4, D)):
            z = x - o
            got = _f(fn, x, o)
            if fn == "griewank":
                want = _mp_griewank(z)
                tol = 64 * EPS * (1 + float((z * z).sum()) / 4000) + D * 4 * EPS * (1 + 600 / 1)
            elif fn == "schwefel":
                want = _mp_schwefel(z)
                tol = 64 * EPS * (418.9829 * D + float(np.abs(z).sum())) + D * 1e-13 * 25
            else:
                want = _mp_powell(z)
                tol = 64 * EPS * float(want) + 1e-300
            assert abs(got - float(want)) <= tol, (fn, D, got, float(want))


def test_griewank_hand_values():
    """z_j = 2 pi k sqrt(j + 1): every cosine is 1, f = sum z^2 / 4000 (up to
    the rounding of z); a single z_0 = pi: cos = -1, f = 2 + pi^2 / 4000."""
    o = np.zeros(1)
    got = _f("griewank", np.array([np.pi]), o)
    assert abs(got - (2 + np.pi**2 / 4000)) <= 1e-13
    D = 6
    z = np.array([2 * np.pi * 3 * np.sqrt(j + 1) for j in range(D)])
    want = float((z * z).sum() / 4000)
    assert abs(_f("griewank", z, np.zeros(D)) - want) <= 1e-11


def test_powell_hand_values():
    """Blocks of 4: (1, 1, 1, 1) -> 121 + 0 + 1 + 0 = 122; (3, -1, 0, 1) ->
    49 + 5 + 1 + 160 = 215; a trailing partial block (z4, 0, 0, 0) -> z4^2 + 10 z4^4."""
    o8 = np.zeros(8)
    assert _f("powell", np.array([1, 1, 1, 1, 3, -1, 0, 1.0]), o8) == 122 + 215
    assert _f("powell", np.array([1, 1, 1, 1, 2.0]), np.zeros(5)) == 122 + (4 + 10 * 16)


def test_schwefel_minimum():
    """z_j = 420.9687 (the function's minimiser to 7 digits): the value is
    D (418.9829 - 420.9687 sin(sqrt(420.9687))), about 1.27e-5 D."""
    D = 10
    z = np.full(D, 420.9687)
    want = float(_mp_schwefel(z))
    assert abs(_f("schwefel", z, np.zeros(D)) - want) <= 1e-9
    assert 0 < want < 2e-4
