"""Pins for the oracle's K_nu (the special function of Eq. 2, Section 2.2).

The oracle integrates K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
(DLMF 10.32.9) with the trapezoidal rule.  These tests tie it to facts that do
not depend on that code: closed forms at half-integer order (DLMF 10.39.2,
10.49.12), SciPy's independent AMOS/Cephes routine, the recurrence
(DLMF 10.29.1), the Wronskian with I_nu from its own power series
(DLMF 10.28.2, 10.25.2), symmetry in nu (DLMF 10.27.3) and the small-x
behaviour (DLMF 10.30.2, 10.31).
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle

XS = np.concatenate([np.logspace(-5, 0, 25), np.linspace(1.1, 60, 30), [100.0, 300.0, 650.0]])


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


def test_half_integer_closed_forms():
    xs = XS[XS < 700]
    k_half = np.sqrt(np.pi / (2 * xs)) * np.exp(-xs)
    assert _rel(oracle.bessel_k(0.5, xs), k_half).max() < 1e-13
    assert _rel(oracle.bessel_k(1.5, xs), k_half * (1 + 1 / xs)).max() < 1e-13
    assert _rel(oracle.bessel_k(2.5, xs), k_half * (1 + 3 / xs + 3 / xs ** 2)).max() < 1e-13


@pytest.mark.parametrize("nu", [0.05, 0.3, 0.7, 1.0, 1.3, 2.0, 3.7, 5.0])
def test_against_scipy(nu):
    got = oracle.bessel_k_scaled(nu, XS)
    want = sp.kve(nu, XS)
    assert _rel(got, want).max() < 2e-13


@pytest.mark.parametrize("nu", [0.7, 1.3, 2.2])
def test_recurrence(nu):
    xs = np.logspace(-2, 1.7, 30)
    km, k0, kp = (oracle.bessel_k(v, xs) for v in (nu - 1, nu, nu + 1))
    assert _rel(km + (2 * nu / xs) * k0, kp).max() < 1e-13


def _bessel_i_series(nu, x, terms=80):
    s, term = 0.0, (x / 2) ** nu / math.gamma(nu + 1)
    for k in range(terms):
        s += term
        term *= (x * x / 4) / ((k + 1) * (k + 1 + nu))
    return s


@pytest.mark.parametrize("nu", [0.3, 0.5, 1.3, 2.7])
def test_wronskian(nu):
    for x in [0.05, 0.3, 1.0, 2.5, 6.0, 10.0]:
        i0, i1 = _bessel_i_series(nu, x), _bessel_i_series(nu + 1, x)
        k0, k1 = oracle.bessel_k(nu, x), oracle.bessel_k(nu + 1, x)
        assert abs((i0 * k1 + i1 * k0) * x - 1.0) < 1e-13


def test_symmetry_in_order():
    xs = np.logspace(-3, 1.5, 12)
    assert _rel(oracle.bessel_k(-0.3, xs), oracle.bessel_k(0.3, xs)).max() == 0.0


@pytest.mark.parametrize("nu", [0.2, 0.45, 0.8])
def test_small_x_two_terms(nu):
    # x^nu K_nu(x) = 2^(nu-1) Gamma(nu) [1 - (x/2)^(2 nu) Gamma(1-nu)/Gamma(1+nu)] + O(x^2)
    x = 1e-4
    lead = 2 ** (nu - 1) * math.gamma(nu)
    two = lead * (1 - (x / 2) ** (2 * nu) * math.gamma(1 - nu) / math.gamma(1 + nu))
    got = x ** nu * oracle.bessel_k(nu, x)
    assert abs(got - two) / two < 1e-7


@pytest.mark.parametrize("nu", [1.3, 2.5, 4.0])
def test_small_x_leading(nu):
    x = 1e-6
    lead = 2 ** (nu - 1) * math.gamma(nu)
    assert abs(x ** nu * oracle.bessel_k(nu, x) - lead) / lead < 1e-10


def test_step_converged():
    for nu in (0.4, 1.3, 3.1):
        for x in (0.01, 0.7, 4.0, 40.0):
            a = oracle.bessel_k_scaled(nu, x, 0.05)
            b = oracle.bessel_k_scaled(nu, x, 0.025)
            assert abs(a - b) / b < 4e-15  # rounding of the longer sum
