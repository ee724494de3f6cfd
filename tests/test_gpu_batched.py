"""Batched evaluation of uneven independent problems (FP64).

Each problem's l must equal the single-problem egs_loglik_ex result bitwise
(same tile size: the batch runs the same device routines in the same order)
and the oracle within the FP64 bar 1e-10; a problem that is not positive
definite is flagged without disturbing the others; a second run of the same
plan replays the captured CUDA graph and gives identical values.
"""
import numpy as np
import pytest

import egs_inputs as ei
import oracle

pytestmark = pytest.mark.gpu

SIZES = [100, 257, 700, 64, 1500, 1, 2, 333, 1024, 1025, 900, 2000]


@pytest.fixture(scope="module")
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    return m


def _problems():
    rng = np.random.default_rng(5)
    out = []
    for k, n in enumerate(SIZES):
        th = (float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.03, 0.12)), float(rng.uniform(0.3, 0.9)))
        p = ei.Problem(n=n, theta=th, seed=100 + k, origin=(0.1, 0.2), side=0.7)
        locs = p.locations()
        z = oracle.simulate_z(locs, th, p.e()) if n > 1 else p.e()
        out.append((n, th, locs, z))
    return out


def test_batched_matches_single_and_oracle(egs):
    from gpu_util import locs_dev, dev
    probs = _problems()
    tile = 128
    B = egs.egs_batch([p[0] for p in probs], tile=tile)
    dl = [locs_dev(p[2]) for p in probs]
    dz = [dev(p[3]) for p in probs]
    thetas = np.array([p[1] for p in probs])
    out, stat = B.run(dl, dz, thetas)
    assert np.all(stat == 0)
    for i, (n, th, locs, z) in enumerate(probs):
        single, _ = egs.egs_loglik_ex(dl[i], dz[i], th, n, "fp64", tile=tile)
        assert out[i] == single, (i, out[i], single)
        ref = oracle.loglik(locs, z, th)["loglik"]
        assert abs(out[i] - ref) <= 1e-10 * max(1.0, abs(ref)), (i, out[i], ref)
    out2, _ = B.run(dl, dz, thetas)            # graph replay
    assert np.array_equal(out, out2)
    assert 0 < B.launches < 2000
    # host inputs give the same values
    out3, _ = B.run([np.ascontiguousarray(p[2].reshape(-1)) for p in probs], [p[3] for p in probs], thetas)
    assert np.array_equal(out, out3)
    B.close()


def test_batched_not_pd_is_isolated(egs):
    from gpu_util import locs_dev, dev
    good = ei.Problem(n=500, theta=(1.0, 0.1, 0.5), seed=1)
    bad_locs = ei.jittered_grid(600, seed=1)
    locs = [good.locations(), bad_locs]
    z = [good.e(), np.ones(600)]
    thetas = [(1.0, 0.1, 0.5), (1.0, 5.0, 4.2)]   # the second is singular in FP64
    out, stat = egs.egs_loglik_batched([locs_dev(l) for l in locs], [dev(v) for v in z], thetas, [500, 600])
    assert stat[0] == 0 and stat[1] == egs.EGS_ERR_NOT_PD
    assert np.isnan(out[1])
    ref = oracle.loglik(locs[0], z[0], thetas[0])["loglik"]
    assert abs(out[0] - ref) <= 1e-10 * abs(ref)


def test_batched_fp32_mode_matches_oracle(egs):
    """FP32-off-band batch (FP64 band of 2 tiles, FP32 off-band tiles and
    updates, FP64 band updates, one FP64 refinement step) on the same uneven
    problems: every l within the FP32-mode bar 1e-6 of the oracle; problems of
    at most 2 tiles are all-FP64; a replay of the graph is bitwise equal."""
    from gpu_util import locs_dev, dev
    probs = _problems()
    B = egs.egs_batch([p[0] for p in probs], tile=128, precision="fp32")
    dl = [locs_dev(p[2]) for p in probs]
    dz = [dev(p[3]) for p in probs]
    thetas = np.array([p[1] for p in probs])
    out, stat = B.run(dl, dz, thetas)
    assert np.all(stat == 0), stat
    worst = 0.0
    for i, (n, th, locs, z) in enumerate(probs):
        ref = oracle.loglik(locs, z, th)["loglik"]
        rel = abs(out[i] - ref) / max(1.0, abs(ref))
        worst = max(worst, rel)
        assert rel <= 1e-6, (i, n, rel)
    print("fp32 batch worst rel l %.2e" % worst)
    out2, _ = B.run(dl, dz, thetas)
    assert np.array_equal(out, out2)
    B.close()
