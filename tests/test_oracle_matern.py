"""Pins for the oracle's Matern covariance (Eq. 2, Section 2.2) and Sigma."""
import math

import numpy as np
import pytest
import scipy.special as sp

import egs_inputs as ei
import oracle


def test_zero_distance_is_variance():
    for th in [(1.0, 0.1, 0.5), (2.5, 0.3, 1.3), (0.7, 1.0, 3.2)]:
        assert oracle.matern(th, 0.0) == th[0]


def test_exponential_and_whittle_special_cases():
    r = np.linspace(0.001, 1.0, 40)
    th = (1.7, 0.13, 0.5)
    assert np.allclose(oracle.matern(th, r), th[0] * np.exp(-r / th[1]), rtol=1e-13, atol=0)
    th = (0.8, 0.2, 1.0)
    x = r / th[1]
    assert np.allclose(oracle.matern(th, r), th[0] * x * sp.kv(1, x), rtol=2e-13, atol=0)


def test_three_halves_closed_form():
    # From Eq. 2 with K_{3/2}(x) = sqrt(pi/2x) e^-x (1 + 1/x): C = theta1 (1 + x) e^-x
    r = np.linspace(0.001, 1.0, 40)
    th = (1.3, 0.09, 1.5)
    x = r / th[1]
    assert np.allclose(oracle.matern(th, r), th[0] * (1 + x) * np.exp(-x), rtol=1e-13, atol=0)


def test_continuity_at_zero():
    th = (1.0, 0.1, 1.3)
    assert abs(oracle.matern(th, 1e-9) - th[0]) < 1e-8


def test_decreasing_in_distance():
    for th in [(1.0, 0.1, 0.5), (1.0, 0.2, 1.3), (1.0, 0.05, 2.2)]:
        v = oracle.matern(th, np.linspace(0.0, 1.4, 200))
        assert np.all(np.diff(v) <= 0)


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.2, 1.3), (1.5, 0.05, 0.9)])
def test_sigma_symmetric_positive_definite(theta):
    locs = ei.jittered_grid(400, seed=2)
    S = oracle.cov_matrix(locs, theta)
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) == theta[0])
    L = oracle.cholesky(S)            # raises if not PD (Section 2: Sigma is SPD)
    assert np.all(np.diag(L) > 0)
    assert np.linalg.eigvalsh(S).min() > 0


def test_cross_covariance_matches_matrix():
    locs = ei.jittered_grid(50, seed=3)
    th = (1.0, 0.2, 1.3)
    S = oracle.cov_matrix(locs, th)
    C = oracle.cov_cross(locs[:, :20], locs, th)
    assert np.array_equal(C, S[:20])
