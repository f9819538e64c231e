"""Pins for the oracle's own sin(pi x) and expm1: mpmath at 300 bits."""
import math

import mpmath
import numpy as np
import pytest

import oracle

mpmath.mp.prec = 300


def _ulp_err(got, exact):
    exact_f = float(exact)
    if exact_f == 0.0:
        return abs(got) / 5e-324
    return float(abs(mpmath.mpf(got) - exact) / mpmath.mpf(np.spacing(abs(exact_f))))


def test_sinpi_special_values():
    for n in range(-8, 9):
        assert oracle.sinpi(float(n)) == 0.0
    assert abs(oracle.sinpi(0.5) - 1.0) <= 2.0**-52
    assert abs(oracle.sinpi(-0.5) + 1.0) <= 2.0**-52
    assert abs(oracle.sinpi(1.0 / 6.0) - 0.5) <= 2.0**-52
    assert oracle.sinpi(1.5) < 0 and oracle.sinpi(2.5) > 0     # (-1)^n sign


def test_sinpi_accuracy():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-0.5, 0.5, 400), rng.uniform(-200, 200, 400),
                         np.array([1e-300, 1e-20, 0.25, 0.49999999999999994, 3.0 + 1e-9,
                                   -7.000000001, 2.0**40 + 0.5])])
    worst = 0.0
    for x in xs:
        exact = mpmath.sin(mpmath.pi * mpmath.mpf(float(x)))
        worst = max(worst, _ulp_err(oracle.sinpi(float(x)), exact))
    assert worst <= 3.0, worst


def test_expm1_special_values():
    assert oracle.expm1(0.0) == 0.0
    assert math.copysign(1.0, oracle.expm1(-0.0)) == -1.0
    assert oracle.expm1(1e-300) == 1e-300
    assert abs(oracle.expm1(-50.0) + 1.0) <= 2.0**-52


def test_expm1_accuracy():
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.uniform(-0.35, 0.35, 300), rng.uniform(-20, 5, 300),
                         np.array([0.3465735902799726, 0.34657359027997264, -0.35, 1e-12,
                                   -1e-12, -13.1, -2.0, 2.0**-30])])
    worst = 0.0
    for x in xs:
        exact = mpmath.expm1(mpmath.mpf(float(x)))
        worst = max(worst, _ulp_err(oracle.expm1(float(x)), exact))
    assert worst <= 3.0, worst
