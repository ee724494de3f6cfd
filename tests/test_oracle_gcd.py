"""Pins of the oracle's great-circle distance (Section 7.4, haversine on
(longitude, latitude) in degrees, sphere of 6371 km): arcs of known angle,
symmetry, and agreement with the local flat-earth approximation at small
separations; the covariance built on it is symmetric positive definite."""
import math

import numpy as np
import pytest

import egs_inputs as ei
import oracle

R = oracle.EARTH_RADIUS_KM


@pytest.mark.parametrize("a,b,angle_deg", [
    ((0.0, 0.0), (0.0, 90.0), 90.0),      # equator to pole
    ((0.0, 0.0), (90.0, 0.0), 90.0),      # along the equator
    ((-40.0, 0.0), (140.0, 0.0), 180.0),  # antipodal on the equator
    ((10.0, 20.0), (10.0, 35.0), 15.0),   # along a meridian
    ((25.0, -10.0), (25.0, -10.0), 0.0),
])
def test_known_arcs(a, b, angle_deg):
    d = oracle.gcd_dist(np.array([[a[0]], [a[1]]]), np.array([[b[0]], [b[1]]]))[0, 0]
    assert abs(d - R * math.radians(angle_deg)) <= 1e-9 * R


def test_symmetric_and_flat_earth_limit():
    locs = ei.jittered_grid(64, seed=3, origin=(-95.0, 30.0), side=0.2)   # ~20 km box
    d = oracle.gcd_dist(locs, locs)
    assert np.allclose(d, d.T, rtol=0, atol=1e-9)
    lam, phi = np.radians(locs[0]), np.radians(locs[1])
    pm = 0.5 * (phi[:, None] + phi[None, :])
    flat = R * np.sqrt((phi[:, None] - phi[None, :]) ** 2 + (np.cos(pm) * (lam[:, None] - lam[None, :])) ** 2)
    off = ~np.eye(64, dtype=bool)
    assert np.max(np.abs(d[off] - flat[off]) / flat[off]) < 1e-6


def test_gcd_covariance_is_spd():
    locs = ei.jittered_grid(100, seed=4, origin=(-95.0, 30.0), side=10.0)
    S = oracle.cov_matrix_gcd(locs, (1.0, 150.0, 0.8))
    assert np.allclose(S, S.T) and np.all(np.diag(S) == 1.0)
    assert np.min(np.linalg.eigvalsh(S)) > 0
