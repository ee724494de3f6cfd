"""IND approximation (Section 6.8) on the GPU against the oracle's
definition (Sigma with the off-diagonal super tiles zeroed): FP64 bar
|dl|/|l| <= 1e-10, ragged last blocks, host and device inputs, and the one-
block case equal to the exact FP64 evaluation (same tile, same device
routines in the same order, so bitwise)."""
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


def _case(n, theta, seed):
    p = ei.Problem(n=n, theta=theta, seed=seed)
    locs = p.locations()
    return locs, oracle.simulate_z(locs, theta, p.e())


@pytest.mark.parametrize("n,tile,super_tiles,theta", [
    (3000, 128, 2, (1.0, 0.1, 0.5)),
    (1000, 64, 3, (1.5, 0.05, 1.2)),    # ragged: 5 blocks of 192 and one of 40
    (2048, 256, 1, (0.8, 0.2, 0.7)),
])
def test_ind_matches_oracle(egs, n, tile, super_tiles, theta):
    from gpu_util import locs_dev, dev
    locs, z = _case(n, theta, 8)
    ref = oracle.loglik_ind(locs, z, theta, tile * super_tiles)
    ll, info = egs.egs_loglik_ind(locs_dev(locs), dev(z), theta, n, tile=tile, super_tiles=super_tiles)
    rel = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    print("IND n=%d tile=%d s=%d rel %.2e" % (n, tile, super_tiles, rel))
    assert rel <= 1e-10
    assert abs(info["logdet"] - ref["logdet"]) <= 1e-10 * abs(ref["logdet"])
    assert info["band"] == super_tiles and info["tile"] == tile


def test_ind_host_inputs_and_single_block(egs):
    from gpu_util import locs_dev, dev
    n, theta = 700, (1.0, 0.1, 0.5)
    locs, z = _case(n, theta, 9)
    a, _ = egs.egs_loglik_ind(locs_dev(locs), dev(z), theta, n, tile=128, super_tiles=2)
    b, _ = egs.egs_loglik_ind(np.ascontiguousarray(locs.reshape(-1)), np.ascontiguousarray(z), theta, n, tile=128,
                              super_tiles=2)
    assert a == b
    one, _ = egs.egs_loglik_ind(locs_dev(locs), dev(z), theta, n, tile=128, super_tiles=6)
    exact, _ = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp64", tile=128)
    assert one == exact
