"""The seeded input generators (egs_inputs): SplitMix64 against its published
outputs, counter-mode stream properties, the distributions drawn from it, the
jittered grid of the paper's synthetic workload (Section 7.1) and the batched
and serving workload recipes."""
import math
from pathlib import Path

import numpy as np

import egs_inputs as ei

GOLDEN = Path(__file__).parent / "golden"


def test_splitmix64_matches_its_published_outputs():
    want = [int(l, 16) for l in (GOLDEN / "splitmix64_state0.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    got = ei._mix64(np.arange(1, 5, dtype=np.uint64) * ei.GOLDEN)
    assert [int(v) for v in got] == want


def test_streams_are_deterministic_and_offsettable():
    a = ei.raw_u64(7, ei.TAG_NORMAL, 100)
    assert np.array_equal(a, ei.raw_u64(7, ei.TAG_NORMAL, 100))
    assert np.array_equal(a[40:60], ei.raw_u64(7, ei.TAG_NORMAL, 20, offset=40))
    assert not np.array_equal(a, ei.raw_u64(7, ei.TAG_BATCH, 100))     # tags are separate streams
    assert not np.array_equal(a, ei.raw_u64(8, ei.TAG_NORMAL, 100))    # and so are seeds
    assert len(set(int(v) for v in a)) == 100


def test_uniform_and_normal_moments():
    u = ei.uniform(3, ei.TAG_BATCH, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    z = ei.normal(3, 200_001)
    assert z.size == 200_001 and np.all(np.isfinite(z))
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / z.size)
    assert abs(np.mean(z ** 4) - 3.0) < 0.1                             # Gaussian kurtosis


def test_jittered_grid_follows_the_synthetic_workload():
    for n in (1600, 1000):
        m = math.isqrt(n) + (0 if math.isqrt(n) ** 2 == n else 1)
        locs = ei.jittered_grid(n, seed=5)
        assert locs.shape == (2, n)
        assert locs.min() > 0.0 and locs.max() < 1.0
        idx = np.arange(n)
        cx = ((idx // m) + 1 - 0.5) / m
        cy = ((idx % m) + 1 - 0.5) / m
        # every point stays within 0.4 / m of its cell centre (X, Y ~ U(-0.4, 0.4) / m)
        assert np.max(np.abs(locs[0] - cx)) <= 0.4 / m and np.max(np.abs(locs[1] - cy)) <= 0.4 / m
        # so no two points coincide: the minimum distance is at least 0.2 / m
        d = np.hypot(locs[0][:, None] - locs[0][None, :], locs[1][:, None] - locs[1][None, :])
        np.fill_diagonal(d, np.inf)
        assert d.min() >= 0.2 / m - 1e-15


def test_batched_and_serving_recipes():
    probs = ei.batched_problems(512)
    ns = np.array([p.n for p in probs])
    assert ns.min() >= 256 and ns.max() <= 4096 and abs(ns.mean() - 2176) < 100
    for p in probs:
        t1, t2, t3 = p.theta
        assert 0.5 <= t1 <= 2.0 and 0.03 <= t2 <= 0.3 and 0.3 <= t3 <= 2.0
        assert 0.2 <= p.side <= 1.0 and 0.0 <= p.origin[0] <= 1.0 - p.side + 1e-12
    fields = ei.serving_fields(64)
    nf = np.array([f.n for f in fields])
    assert nf.min() >= 1000 and nf.max() <= 40000
    assert abs(np.mean(np.log(nf)) - 0.5 * (math.log(1000) + math.log(40000))) < 0.4
