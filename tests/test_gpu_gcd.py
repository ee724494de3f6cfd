"""Great-circle distance (Section 7.4) in the Matern generator: the FP64
log-likelihood on (longitude, latitude) locations in a 10 x 10 degree box
(about the size of the paper's soil-moisture region) against the oracle
built on its own haversine distances: |dl|/|l| <= 1e-10."""
import numpy as np
import pytest

import egs_inputs as ei
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    return m


@pytest.mark.parametrize("n,theta,tile", [(1600, (1.0, 100.0, 0.5), 320), (2000, (1.3, 60.0, 1.2), 256)])
def test_gcd_loglik_matches_oracle(egs, n, theta, tile):
    from gpu_util import locs_dev, dev
    locs = ei.jittered_grid(n, seed=21, origin=(-95.0, 30.0), side=10.0)
    S = oracle.cov_matrix_gcd(locs, theta)
    z = np.linalg.cholesky(S) @ ei.normal(21, n)
    ref = oracle.loglik_gcd(locs, z, theta)
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp64", tile=tile, distance="great_circle")
    rel = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    print("gcd n=%d rel %.2e" % (n, rel))
    assert rel <= 1e-10
    # the same coordinates read as Euclidean degrees give a different model
    # (with theta2 in km that matrix is numerically singular or far off)
    try:
        le, _ = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp64", tile=tile)
    except egs.NotPositiveDefinite:
        return
    assert abs(le - ll) > 1e-3 * abs(ll)


def test_gcd_fp32_mode_matches_oracle(egs):
    """The FP32 mixed mode under the great-circle distance: the generator and
    the refinement residual take the direct FP64 evaluation (the double-float
    path covers the Euclidean distance only); l within the FP32-mode bar of
    the oracle, and several refinement steps bring the quadratic form to the
    FP64 bar."""
    from gpu_util import locs_dev, dev
    n, theta = 3000, (1.0, 80.0, 0.5)
    locs = ei.jittered_grid(n, seed=22, origin=(-95.0, 30.0), side=10.0)
    S = oracle.cov_matrix_gcd(locs, theta)
    z = np.linalg.cholesky(S) @ ei.normal(22, n)
    ref = oracle.loglik_gcd(locs, z, theta)
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp32", tile=256, band=2,
                                 distance="great_circle")
    rel = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    _, i4 = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp32", tile=256, band=2, refine=4,
                              distance="great_circle")
    q4 = abs(i4["quad"] - ref["quad"]) / ref["quad"]
    print("gcd fp32 n=%d rel l %.2e, quad after 4 refinement steps %.2e" % (n, rel, q4))
    assert rel <= 1e-6
    assert q4 <= 1e-10
