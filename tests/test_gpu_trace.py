"""The per-launch trace (egs_opts.timing = 3): one record per launch the call
counted, stream-ordered records that do not overlap on their stream, class
totals equal to the per-class sums the call reports, and the lookahead chain
(diagonal POTRF) on the side stream of the mixed factorisation."""
import numpy as np
import pytest

import egs_inputs as ei

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    return m


@pytest.mark.parametrize("prec,tile,band", [("fp64", 256, 0), ("fp32", 256, 2)])
def test_trace_matches_the_call(egs, prec, tile, band):
    from gpu_util import locs_dev, dev
    n, theta = 3000, (1.0, 0.1, 0.5)
    p = ei.Problem(n=n, theta=theta, seed=5)
    locs = p.locations()
    z = p.e()
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=tile, band=band, timing=3)
    tr = egs.egs_trace_last()
    assert len(tr) == info["launches"] > 0
    T = -(-n // tile)
    assert tr[0][0] == "generate"
    for cls, step, stream, t0, t1 in tr:
        assert 0.0 <= t0 <= t1 <= info["ms_total"] + 0.05
        assert -1 <= step < T and stream in (0, 1)
    for st in (0, 1):
        rows = [r for r in tr if r[2] == st]
        for a, b in zip(rows, rows[1:]):
            assert b[3] >= a[4] - 1e-3      # one stream runs its launches in order
    for cls, key in (("potrf", "ms_potrf"), ("trsm", "ms_trsm"), ("update", "ms_update"), ("solve", "ms_trsv")):
        tot = sum(r[4] - r[3] for r in tr if r[0] == cls)
        assert abs(tot - info[key]) <= 1e-3 * max(1.0, info[key]) + 0.01
    steps = {r[1] for r in tr if r[0] == "potrf"}
    assert steps == set(range(T))
    side = [r for r in tr if r[2] == 1]
    if prec == "fp64":
        assert not side
    else:
        assert side and {r[0] for r in side} >= {"potrf"}
    # a call without timing = 3 leaves the trace of the last traced call alone
    egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=tile, band=band)
    assert len(egs.egs_trace_last()) == len(tr)
