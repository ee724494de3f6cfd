"""Pins of the oracle's kriging prediction (Eq. 5, Algorithm 3):
closed forms for one and two observed locations with the exponential model
(nu = 1/2, C(r) = theta1 exp(-r / theta2)), the interpolation property (no
nugget: predicting at an observed location returns its measurement),
linearity in Z_2 and the far-field limit."""
import math

import numpy as np
import pytest

import egs_inputs as ei
import oracle


def test_one_observed_location_closed_form():
    theta = (2.0, 0.3, 0.5)
    obs = np.array([[0.2], [0.3]])
    new = np.array([[0.5, 0.2, 0.9], [0.7, 0.3, 0.1]])
    z2 = np.array([1.7])
    got = oracle.predict(obs, z2, new, theta)
    r = np.hypot(new[0] - 0.2, new[1] - 0.3)
    want = np.exp(-r / 0.3) * 1.7          # C(r) / C(0) * z
    assert np.allclose(got, want, rtol=1e-13, atol=0)


def test_two_observed_locations_closed_form():
    theta = (1.3, 0.2, 0.5)
    obs = np.array([[0.1, 0.4], [0.2, 0.25]])
    new = np.array([[0.3], [0.6]])
    z2 = np.array([0.8, -1.1])
    a = 1.3
    c = 1.3 * math.exp(-math.hypot(0.3, 0.05) / 0.2)
    k1 = 1.3 * math.exp(-math.hypot(0.2, 0.4) / 0.2)
    k2 = 1.3 * math.exp(-math.hypot(0.1, 0.35) / 0.2)
    det = a * a - c * c                     # [[a, c], [c, a]]^-1 = [[a, -c], [-c, a]] / det
    x = np.array([a * 0.8 - c * -1.1, -c * 0.8 + a * -1.1]) / det
    want = k1 * x[0] + k2 * x[1]
    got = oracle.predict(obs, z2, new, theta)
    assert abs(got[0] - want) <= 1e-13 * abs(want)


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.5, 0.05, 1.2)])
def test_interpolates_observed_measurements(theta):
    p = ei.Problem(n=200, theta=theta, seed=3)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    got = oracle.predict(locs, z, locs[:, ::7], theta)
    assert np.max(np.abs(got - z[::7])) <= 1e-8 * np.max(np.abs(z))


def test_linear_in_z_and_vanishes_far_away():
    theta = (1.0, 0.05, 0.8)
    p = ei.Problem(n=150, theta=theta, seed=4)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    new = np.array([[0.33, 0.71, 40.0], [0.52, 0.18, 40.0]])
    a = oracle.predict(locs, z, new, theta)
    b = oracle.predict(locs, 2.5 * z, new, theta)
    assert np.allclose(b, 2.5 * a, rtol=1e-12, atol=1e-15)
    assert abs(a[2]) < 1e-200                # ~800 ranges away: C(r) underflows
