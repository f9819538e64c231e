"""Pins for the oracle's fitness functions (Table 3.2, shifted / rotated forms).

Closed forms at hand-computed points, rotation invariance, and an mpmath
evaluation of each function's textbook definition (cos, exp -- not the
identities the oracle uses) at random points."""
import math

import mpmath
import numpy as np
import pytest

import oracle
import workload

mpmath.mp.prec = 200
EPS = 2.0**-53


def _o(D, seed=5):
    return workload.shift(D, -3.0, 3.0, seed)


@pytest.mark.parametrize("D", [1, 2, 5, 30, 100, 257])
def test_closed_forms(D):
    o = _o(D)
    w = workload.ellipsoid_weights(D)
    assert oracle.fitness("sphere", o, o) == 0.0
    assert oracle.fitness("rastrigin", o, o) == 0.0
    assert oracle.fitness("ackley", o, o) == 0.0
    assert oracle.fitness("rosenbrock", o, o) == 0.0
    assert oracle.fitness("ellipsoid", o, o, w) == 0.0
    one = np.ones(D)
    # Sphere at o + 1: D.  Rastrigin at integer offsets: sum of squares (sin^2(pi k) = 0).
    x = o + one
    tol = 8 * D * EPS * D
    assert abs(oracle.fitness("sphere", x, o) - D) <= tol
    ks = np.arange(D) % 5 - 2.0
    assert abs(oracle.fitness("rastrigin", o + ks, o) - float((ks**2).sum())) <= 1e-9 * max(1, D)
    # Rastrigin at o + 1/2: D (1/4 + 20).
    assert abs(oracle.fitness("rastrigin", o + 0.5, o) - D * 20.25) <= 1e-12 * D * 20.25 + 1e-9
    # Rosenbrock at x = o - 1 (a = 0): every term is (0 - 1)^2 = 1 -> D - 1.
    assert abs(oracle.fitness("rosenbrock", o - 1.0, o) - (D - 1)) <= 1e-12 * D
    # Ackley at integer offsets 1: S1 = D, cos = 1 -> 20 (1 - e^-0.2).
    expect = 20.0 * (1.0 - math.exp(-0.2))
    assert abs(oracle.fitness("ackley", o + 1.0, o) - expect) <= 1e-13
    # Ellipsoid: unit step in coordinate k gives w_k.
    for k in {0, D // 2, D - 1}:
        e = np.zeros(D)
        e[k] = 1.0
        assert abs(oracle.fitness("ellipsoid", o + e, o, w) - w[k]) <= 4 * EPS * w[k]


def _exact(fn, x, o, w=None, M=None):
    D = len(x)
    d = [mpmath.mpf(float(a)) - mpmath.mpf(float(b)) for a, b in zip(x, o)]
    if M is not None:
        z = [mpmath.fsum(mpmath.mpf(float(M[j, k])) * d[k] for k in range(D)) for j in range(D)]
    else:
        z = d
    base = fn.replace("rot_", "")
    pi = mpmath.pi
    if base == "sphere":
        return mpmath.fsum(v * v for v in z)
    if base == "ellipsoid":
        return mpmath.fsum(mpmath.mpf(float(w[j])) * z[j] ** 2 for j in range(D))
    if base == "rastrigin":
        return 10 * D + mpmath.fsum(v * v - 10 * mpmath.cos(2 * pi * v) for v in z)
    if base == "rosenbrock":
        a = [v + 1 for v in z]
        return mpmath.fsum(100 * (a[j + 1] - a[j] ** 2) ** 2 + (a[j] - 1) ** 2
                           for j in range(D - 1))
    if base == "ackley":
        s1 = mpmath.fsum(v * v for v in z) / D
        s2 = mpmath.fsum(mpmath.cos(2 * pi * v) for v in z) / D
        return -20 * mpmath.exp(-0.2 * mpmath.sqrt(s1)) - mpmath.exp(s2) + 20 + mpmath.e
    raise KeyError(fn)


@pytest.mark.parametrize("fn", ["sphere", "ellipsoid", "rastrigin", "rosenbrock", "ackley",
                                "rot_ellipsoid", "rot_rastrigin", "rot_ackley"])
@pytest.mark.parametrize("D", [1, 3, 17, 64])
def test_textbook_definition(fn, D):
    lb, ub = workload.BOUNDS[fn]
    rng = np.random.default_rng(D * 31 + len(fn))
    o = workload.shift(D, 0.8 * lb, 0.8 * ub, 2)
    w = workload.ellipsoid_weights(D)
    M = workload.rotation(D, 3) if fn.startswith("rot_") else None
    for _ in range(4):
        x = rng.uniform(lb, ub, D)
        got = oracle.fitness(fn, x, o, w, M)
        exact = _exact(fn, x, o, w, M)
        # FP64 evaluation error: a few eps per operation on the magnitude involved.
        scale = float(abs(exact)) + 1.0
        assert abs(mpmath.mpf(got) - exact) <= 1e-12 * scale * (D + 8), (fn, D)


def test_rotation_preserves_norm():
    """M orthogonal: rotated ellipsoid with unit weights equals the sphere."""
    D = 40
    M = workload.rotation(D, 8)
    assert np.abs(M @ M.T - np.eye(D)).max() <= 1e-13
    o = _o(D)
    x = o + np.random.default_rng(1).uniform(-1, 1, D)
    a = oracle.fitness("rot_ellipsoid", x, o, np.ones(D), M)
    b = oracle.fitness("sphere", x, o)
    assert abs(a - b) <= 1e-12 * b


def test_rotated_at_preimage():
    """x = o + M^T v gives z = v (up to rounding): rotated Rastrigin of v = 1/2."""
    D = 24
    M = workload.rotation(D, 9)
    o = _o(D)
    x = o + M.T @ np.full(D, 0.5)
    assert abs(oracle.fitness("rot_rastrigin", x, o, None, M) - 20.25 * D) <= 1e-9 * D


def _fma(a, b, c):
    """Correctly rounded a*b + c via exact rationals (independent of libm)."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


@pytest.mark.parametrize("D", [7, 100, 300])
def test_summation_order_is_fixed(D):
    """The FP64 sum follows the documented order bit for bit: variable j feeds
    lane (j>>2)&31, lanes accumulate fma(z, z, acc) in ascending j from +0.0,
    then an xor butterfly over offsets 16, 8, 4, 2, 1."""
    rng = np.random.default_rng(12 + D)
    z = rng.uniform(-100, 100, D)
    lanes = [0.0] * 32
    for j in range(D):
        l = (j >> 2) & 31
        lanes[l] = _fma(float(z[j]), float(z[j]), lanes[l])
    for off in (16, 8, 4, 2, 1):
        lanes = [lanes[l] + lanes[l ^ off] for l in range(32)]
    got = oracle.fitness("sphere", z, np.zeros(D))
    assert got == lanes[0]
    exact = float(mpmath.fsum(mpmath.mpf(float(v)) ** 2 for v in z))
    assert abs(got - exact) <= 40 * EPS * exact
