"""Pins for the oracle's log-likelihood (Eq. 1 evaluated by Algorithm 2).

Brute force in long double on n <= 64, closed forms for n = 1, 2 and for a
diagonal Sigma, invariances of Eq. 1, agreement of the two independent
factorisations (textbook C Cholesky and LAPACK dpotrf), and a loose
statistical check on data simulated by Algorithm 1.  The "planted mistake"
tests at the end show that a plausible error in the oracle (a dropped factor
2, a sign, a transposed solve) fails these pins.
"""
import math

import numpy as np
import pytest

import egs_inputs as ei
import oracle

LOG2PI = math.log(2 * math.pi)


def _case(n, theta, seed=0):
    p = ei.Problem(n=n, theta=theta, seed=seed)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e()) if n > 1 else p.e()
    return locs, z


def brute_loglik(locs, z, theta):
    S = oracle.cov_matrix(locs, theta)
    sign, logdet = oracle.brute_logdet(S)
    assert sign == 1
    q = oracle.brute_quad(S, z)
    n = len(z)
    return -0.5 * q - 0.5 * logdet - 0.5 * n * LOG2PI, logdet, q


def check_brute(impl):
    for n, th in [(17, (1.0, 0.1, 0.5)), (40, (1.3, 0.2, 1.3)), (64, (0.7, 0.15, 0.8))]:
        locs, z = _case(n, th, seed=n)
        got = impl(locs, z, th)
        ll, ld, q = brute_loglik(locs, z, th)
        assert abs(got["logdet"] - ld) <= 1e-11 * max(1.0, abs(ld))
        assert abs(got["quad"] - q) <= 1e-11 * abs(q)
        assert abs(got["loglik"] - ll) <= 1e-12 * abs(ll)


def check_n1(impl):
    th = (1.7, 0.1, 0.5)
    locs = np.array([[0.3], [0.4]])
    z = np.array([0.9])
    got = impl(locs, z, th)["loglik"]
    want = -0.5 * LOG2PI - 0.5 * math.log(th[0]) - z[0] ** 2 / (2 * th[0])
    assert abs(got - want) < 1e-14


def check_n2(impl):
    th = (1.2, 0.2, 1.3)
    locs = np.array([[0.1, 0.25], [0.3, 0.2]])
    z = np.array([0.7, -0.4])
    r = math.hypot(0.15, 0.1)
    c = float(oracle.matern(th, r))
    det = th[0] ** 2 - c * c
    q = (th[0] * z[0] ** 2 - 2 * c * z[0] * z[1] + th[0] * z[1] ** 2) / det
    want = -LOG2PI - 0.5 * math.log(det) - 0.5 * q
    got = impl(locs, z, th)
    assert abs(got["loglik"] - want) < 1e-13
    assert abs(got["logdet"] - math.log(det)) < 1e-13


def check_diagonal_limit(impl):
    # theta2 -> 0+: all off-diagonal entries underflow, Sigma = theta1 I
    locs, z = _case(200, (1.0, 0.1, 0.5), seed=3)
    th = (2.3, 1e-5, 0.9)
    n = len(z)
    want = -0.5 * n * math.log(2 * math.pi * th[0]) - 0.5 * float(z @ z) / th[0]
    assert abs(impl(locs, z, th)["loglik"] - want) <= 1e-13 * abs(want)


IMPLS = {"c": oracle.loglik, "lapack": oracle.loglik_lapack}


@pytest.mark.parametrize("impl", list(IMPLS))
def test_brute_force(impl):
    check_brute(IMPLS[impl])


@pytest.mark.parametrize("impl", list(IMPLS))
def test_closed_forms(impl):
    check_n1(IMPLS[impl])
    check_n2(IMPLS[impl])
    check_diagonal_limit(IMPLS[impl])


def test_variance_scaling():
    locs, z = _case(300, (1.0, 0.1, 0.7), seed=4)
    th = (1.0, 0.1, 0.7)
    a = oracle.loglik(locs, z, th)
    c = 3.7
    b = oracle.loglik(locs, z, (c, 0.1, 0.7))
    n = len(z)
    want = a["loglik"] - 0.5 * n * math.log(c) - 0.5 * (1 / c - 1) * a["quad"]
    assert abs(b["loglik"] - want) <= 1e-12 * abs(want)


def test_location_range_scaling():
    locs, z = _case(300, (1.0, 0.1, 1.3), seed=5)
    a = oracle.loglik(locs, z, (1.0, 0.1, 1.3))["loglik"]
    b = oracle.loglik(locs * 2.5, z, (1.0, 0.25, 1.3))["loglik"]
    assert abs(a - b) <= 1e-11 * abs(a)


def test_permutation_invariance():
    locs, z = _case(300, (1.0, 0.1, 0.5), seed=6)
    perm = np.random.default_rng(0).permutation(300)
    a = oracle.loglik(locs, z, (1.0, 0.1, 0.5))["loglik"]
    b = oracle.loglik(locs[:, perm], z[perm], (1.0, 0.1, 0.5))["loglik"]
    assert abs(a - b) <= 1e-12 * abs(a)


def test_c_and_lapack_agree():
    for th in [(1.0, 0.1, 0.5), (1.0, 0.2, 1.3)]:
        locs, z = _case(900, th, seed=8)
        a, b = oracle.loglik(locs, z, th), oracle.loglik_lapack(locs, z, th)
        for k in ("loglik", "logdet", "quad"):
            assert abs(a[k] - b[k]) <= 1e-11 * abs(b[k]), k


def test_simulated_quadratic_form_is_chi_square():
    # Algorithm 1: Z = L e with e ~ N(0, I) gives Z^T Sigma^-1 Z = e^T e ~ chi^2_n
    n = 1600
    locs, z = _case(n, (1.0, 0.1, 0.5), seed=0)
    q = oracle.loglik(locs, z, (1.0, 0.1, 0.5))["quad"]
    assert abs(q / n - 1.0) < 5 * math.sqrt(2.0 / n)


def test_not_positive_definite_is_reported():
    locs = ei.jittered_grid(600, seed=1)
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.loglik(locs, np.ones(600), (1.0, 5.0, 4.2))


# ---- planted mistakes: each mutated oracle must fail at least one pin ----

def _mut_logdet_no_factor_two(locs, z, th):
    r = oracle.loglik(locs, z, th)
    r = dict(r)
    r["logdet"] /= 2
    r["loglik"] = -0.5 * r["quad"] - 0.5 * r["logdet"] - 0.5 * len(z) * LOG2PI
    return r


def _mut_quad_sign(locs, z, th):
    r = dict(oracle.loglik(locs, z, th))
    r["loglik"] = 0.5 * r["quad"] - 0.5 * r["logdet"] - 0.5 * len(z) * LOG2PI
    return r


def _mut_transposed_solve(locs, z, th):
    import scipy.linalg as sla
    S = oracle.cov_matrix(locs, th)
    L = np.linalg.cholesky(S)
    y = sla.solve_triangular(L.T, z, lower=False)   # wrong triangle
    ld = 2 * np.sum(np.log(np.diag(L)))
    q = float(y @ y)
    return {"loglik": -0.5 * q - 0.5 * ld - 0.5 * len(z) * LOG2PI, "logdet": ld, "quad": q}


def _mut_range_not_divided(locs, z, th):
    return oracle.loglik(locs, z, (th[0], 1.0, th[2]))


@pytest.mark.parametrize("mut", [_mut_logdet_no_factor_two, _mut_quad_sign, _mut_transposed_solve,
                                 _mut_range_not_divided])
def test_planted_mistakes_are_caught(mut):
    caught = 0
    for check in (check_brute, check_n1, check_n2, check_diagonal_limit):
        try:
            check(mut)
        except AssertionError:
            caught += 1
    assert caught >= 1


@pytest.mark.parametrize("n,th", [(40, (1.3, 0.2, 1.3)), (64, (0.7, 0.15, 0.8))])
def test_simulate_loglik_against_brute_force(n, th):
    """Algorithm 1 then Algorithm 2 on one factorisation: the returned z is
    L e, and l, log|Sigma|, Z^T Sigma^-1 Z match the long-double brute force
    on that z."""
    p = ei.Problem(n=n, theta=th, seed=n)
    locs, e = p.locations(), p.e()
    r = oracle.simulate_loglik(locs, th, e)
    assert np.allclose(r["z"], oracle.simulate_z(locs, th, e), rtol=0, atol=1e-14)
    ll, ld, q = brute_loglik(locs, r["z"], th)
    assert abs(r["logdet"] - ld) <= 1e-11 * max(1.0, abs(ld))
    assert abs(r["quad"] - q) <= 1e-11 * abs(q)
    assert abs(r["loglik"] - ll) <= 1e-12 * abs(ll)
    # Z = L e, so Z^T Sigma^-1 Z = e^T e (Algorithm 1 and Eq. 1 together)
    assert abs(r["quad"] - float(e @ e)) <= 1e-11 * float(e @ e)


def test_simulate_loglik_matches_separate_calls():
    n, th = 900, (1.0, 0.2, 1.3)
    p = ei.Problem(n=n, theta=th, seed=2)
    locs, e = p.locations(), p.e()
    r = oracle.simulate_loglik(locs, th, e)
    z = oracle.simulate_z(locs, th, e)
    ref = oracle.loglik_lapack(locs, z, th)
    for k in ("loglik", "logdet", "quad"):
        assert abs(r[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
