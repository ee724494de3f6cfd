"""Batched evaluation of uneven independent problems (FP64).

FP64 batches run as one persistent launch over the tile-task graph of every
problem.  Each problem's l must equal the single-problem egs_loglik_ex result
bitwise (same tile size: the batch runs the same device routines in the same
order on each tile) and the oracle within the FP64 bar 1e-10; a problem that
is not positive definite is flagged without disturbing the others; a second
run of the same plan replays the captured CUDA graph and gives identical
values.  Failure detection: with a task's completion withheld, the dependency
waits run out, the run reports EGS_ERR_TIMEOUT without hanging, and the next
normal run of the same batch is correct.  The tile autotuner stores its choice
where egs_batch(tile=0) finds it.
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


@pytest.mark.parametrize("tile", [64, 128, 192, 256])
def test_batched_matches_single_and_oracle(egs, tile):
    from gpu_util import locs_dev, dev
    probs = _problems()
    B = egs.egs_batch([p[0] for p in probs], tile=tile)
    assert B.tasks > 0                          # one persistent launch over the task graph
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
    assert B.launches == 2                      # the general-nu polynomials, then the persistent launch
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


def test_batched_wait_timeout_then_recovers(egs):
    """The completion of one task (problem 0's first generated tile) is
    withheld: the waits that need it run out after 2 ms, every CTA stops
    claiming work, and the run returns EGS_ERR_TIMEOUT.  With the hook
    removed, the same batch returns the values of a clean run."""
    from gpu_util import locs_dev, dev
    probs = _problems()
    dl = [locs_dev(p[2]) for p in probs]
    dz = [dev(p[3]) for p in probs]
    thetas = np.array([p[1] for p in probs])
    B = egs.egs_batch([p[0] for p in probs], tile=128)
    want, _ = B.run(dl, dz, thetas)
    B.set_wait_limit(2_000_000, withhold_task=0)
    with pytest.raises(egs.EgsError) as e:
        B.run(dl, dz, thetas)
    assert e.value.status == egs.EGS_ERR_TIMEOUT
    B.set_wait_limit(10_000_000_000, withhold_task=-1)
    got, stat = B.run(dl, dz, thetas)
    assert np.all(stat == 0) and np.array_equal(got, want)
    B.close()


def test_batch_autotuner_table(egs):
    from gpu_util import locs_dev, dev
    probs = _problems()
    ns = [p[0] for p in probs]
    dl = [locs_dev(p[2]) for p in probs]
    dz = [dev(p[3]) for p in probs]
    thetas = np.array([p[1] for p in probs])
    best, ms = egs.egs_batch_autotune(ns, dl, dz, thetas, "fp64")
    assert best in (64, 128, 256) and all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    assert egs.egs_batch_tuned_tile(max(ns), "fp64") == best
    B = egs.egs_batch(ns, tile=0)
    assert B.tile == best
    out, stat = B.run(dl, dz, thetas)
    for i, (n, th, locs, z) in enumerate(probs):
        ref = oracle.loglik(locs, z, th)["loglik"]
        assert abs(out[i] - ref) <= 1e-10 * max(1.0, abs(ref))
    B.close()
