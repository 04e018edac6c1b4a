"""Pins for the oracle's Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt,
the only special function of the ERI (Sec. II.C; [00|00]^(m) seeds).

Each pin is independent of the oracle's series/recursion: closed forms, the
large-T asymptote, adaptive quadrature of the defining integral, and the
agreement of the oracle's two branches where both are valid."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


def test_boys_at_zero():
    F = oracle.boys(12, 0.0)
    for m in range(13):
        assert F[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.1, 0.7, 2.5, 9.0, 17.0, 33.0, 39.9, 40.1, 80.0, 500.0])
def test_boys_f0_closed_form(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert oracle.boys(0, T)[0] == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("T", [45.0, 120.0, 900.0])
def test_boys_asymptote(T):
    F = oracle.boys(10, T)
    for m in range(11):
        dfact = np.prod(np.arange(2 * m - 1, 0, -2)) if m > 0 else 1.0
        ref = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        # e^-T corrections are below 1e-19 relative here
        assert F[m] == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("T", [0.05, 1.0, 6.0, 25.0, 55.0])
def test_boys_quadrature(T):
    F = oracle.boys(11, T)
    for m in range(12):
        ref, err = integrate.quad(lambda t: t ** (2 * m) * math.exp(-T * t * t), 0.0, 1.0,
                                  epsabs=0, epsrel=1e-13, limit=200)
        assert F[m] == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("T", [6.0, 15.0, 30.0, 39.0, 45.0])
def test_boys_branches_agree(T):
    a = oracle.boys(11, T, branch=1)
    b = oracle.boys(11, T, branch=2)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)
