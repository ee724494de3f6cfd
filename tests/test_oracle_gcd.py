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


LOG2PI = math.log(2 * math.pi)


def test_loglik_gcd_n1_closed_form():
    """n = 1: Sigma = theta1, so l = -1/2 log(2 pi) - 1/2 log theta1 - z^2 / (2 theta1)
    whatever the location (Eq. 1)."""
    th = (1.7, 300.0, 0.8)
    locs = np.array([[-92.5], [34.0]])
    z = np.array([0.9])
    got = oracle.loglik_gcd(locs, z, th)
    want = -0.5 * LOG2PI - 0.5 * math.log(th[0]) - z[0] ** 2 / (2 * th[0])
    assert abs(got["loglik"] - want) < 1e-14
    assert abs(got["logdet"] - math.log(th[0])) < 1e-14
    assert abs(got["quad"] - z[0] ** 2 / th[0]) < 1e-14


def test_loglik_gcd_n2_closed_form():
    """n = 2 on one meridian, 15 degrees apart: the great-circle distance is
    R * 15 pi / 180, and with nu = 1/2 the covariance is theta1 exp(-d / theta2)
    (Section 2.2), so |Sigma| = theta1^2 - c^2 and Z^T Sigma^-1 Z are closed
    forms that use neither the oracle's distance nor its Matern."""
    th = (1.2, 2000.0, 0.5)
    locs = np.array([[10.0, 10.0], [20.0, 35.0]])
    z = np.array([0.7, -0.4])
    d = R * math.radians(15.0)
    c = th[0] * math.exp(-d / th[1])
    det = th[0] ** 2 - c * c
    q = (th[0] * z[0] ** 2 - 2 * c * z[0] * z[1] + th[0] * z[1] ** 2) / det
    want = -LOG2PI - 0.5 * math.log(det) - 0.5 * q
    got = oracle.loglik_gcd(locs, z, th)
    assert abs(got["logdet"] - math.log(det)) < 1e-13
    assert abs(got["quad"] - q) < 1e-13 * abs(q)
    assert abs(got["loglik"] - want) < 1e-13


@pytest.mark.parametrize("n,theta", [(17, (1.0, 120.0, 0.5)), (48, (1.3, 250.0, 1.3))])
def test_loglik_gcd_against_brute_force(n, theta):
    """The assembly of l (log-determinant, quadratic form, -n/2 log 2 pi) on
    the great-circle Sigma against a long-double LU determinant and a
    Gauss-Jordan inverse of the same matrix."""
    locs = ei.jittered_grid(n, seed=n, origin=(-95.0, 30.0), side=10.0)
    z = ei.normal(n, n)
    S = oracle.cov_matrix_gcd(locs, theta)
    sign, logdet = oracle.brute_logdet(S)
    assert sign == 1
    q = oracle.brute_quad(S, z)
    want = -0.5 * q - 0.5 * logdet - 0.5 * n * LOG2PI
    got = oracle.loglik_gcd(locs, z, theta)
    assert abs(got["logdet"] - logdet) <= 1e-11 * max(1.0, abs(logdet))
    assert abs(got["quad"] - q) <= 1e-11 * abs(q)
    assert abs(got["loglik"] - want) <= 1e-12 * abs(want)
