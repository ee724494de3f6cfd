"""The bench's algorithmic flop counts (used for the roofline) against a
brute-force enumeration of the tile updates of the right-looking tile
Cholesky: every update C_mn -= P_m P_n^T at step k (T > m >= n > k) costs
b^3 (SYRK, m = n) or 2 b^3 (GEMM), and splits into band x band, other band
outputs (m - n < band) and off-band outputs."""
import pytest

import bench


@pytest.mark.parametrize("n,b,band", [(4096, 512, 2), (5000, 256, 3), (102400, 512, 2), (2048, 512, 4)])
def test_update_flops_partition(n, b, band):
    T = -(-n // b)
    bb = bo = off = 0.0
    for k in range(T):
        for m in range(k + 1, T):
            for c in range(k + 1, m + 1):
                f = b ** 3 if m == c else 2 * b ** 3
                if m - k < band and c - k < band:
                    bb += f
                elif m - c < band:
                    bo += f
                else:
                    off += f
    fc = bench.flop_counts(n, b)
    assert abs(fc["update"] - (bb + bo + off)) <= 1e-9 * fc["update"]
    assert abs(bench.band_band_flops(n, b, band) - bb) <= 1e-9 * max(bb, 1.0)
    assert abs(bench.band_out_flops(n, b, band) - bo) <= 1e-9 * max(bo, 1.0)


def test_timeline_summary_splits_streams_and_idle():
    import bench
    trace = [("generate", -1, 0, 0.0, 5.0),
             ("potrf", 0, 1, 5.0, 6.0), ("trsm", 0, 0, 6.0, 7.0), ("update", 0, 0, 7.0, 9.0),
             ("potrf", 1, 1, 7.5, 8.0), ("trsm", 1, 0, 10.0, 10.5), ("update_f64", 1, 1, 8.0, 9.5),
             ("solve", -1, 0, 10.5, 12.0)]
    t = bench.timeline_summary(trace)
    assert t["factor_span_ms"] == 5.5
    assert t["main_ms"] == {"trsm": 1.5, "update": 2.0}
    assert t["side_ms"] == {"potrf": 1.5, "update_f64": 1.5}
    assert abs(t["main_idle_ms"] - 2.0) < 1e-12
    assert bench.timeline_summary([("generate", -1, 0, 0.0, 1.0)]) == {}
