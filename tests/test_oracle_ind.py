"""Pins of the oracle's IND approximation (Section 6.8: off-diagonal super
tiles set to zero).  A block-diagonal Sigma has log|Sigma| = sum of the
blocks' log-determinants and Z^T Sigma^-1 Z = sum of the blocks' quadratic
forms, so l_IND must equal the sum of the C oracle's l over the blocks (an
independent code path: unblocked C Cholesky per block against LAPACK on the
masked n x n matrix), and a single block must give the exact l."""
import numpy as np
import pytest

import egs_inputs as ei
import oracle


def _case(n, theta=(1.0, 0.1, 0.5), seed=2):
    p = ei.Problem(n=n, theta=theta, seed=seed)
    locs = p.locations()
    return locs, oracle.simulate_z(locs, theta, p.e()), theta


@pytest.mark.parametrize("n,block", [(300, 64), (257, 100), (200, 1), (130, 129)])
def test_ind_is_sum_over_blocks(n, block):
    locs, z, theta = _case(n)
    ind = oracle.loglik_ind(locs, z, theta, block)
    tot = {"loglik": 0.0, "logdet": 0.0, "quad": 0.0}
    for s in range(0, n, block):
        r = oracle.loglik(locs[:, s:s + block], z[s:s + block], theta)
        for k in tot:
            tot[k] += r[k]
    for k in tot:
        assert abs(ind[k] - tot[k]) <= 1e-11 * max(1.0, abs(tot[k])), (k, ind[k], tot[k])


def test_ind_single_block_is_exact():
    locs, z, theta = _case(250)
    full = oracle.loglik(locs, z, theta)
    ind = oracle.loglik_ind(locs, z, theta, 250)
    assert abs(ind["loglik"] - full["loglik"]) <= 1e-11 * abs(full["loglik"])


def test_ind_differs_from_exact_when_blocks_split_correlated_points():
    """The approximation drops real correlations: with range 0.1 on 300
    points the IND value must differ from the exact one (a mask that zeroed
    nothing would pass the sum test above only by accident)."""
    locs, z, theta = _case(300)
    full = oracle.loglik(locs, z, theta)["loglik"]
    ind = oracle.loglik_ind(locs, z, theta, 50)["loglik"]
    assert abs(ind - full) > 1e-3 * abs(full)
