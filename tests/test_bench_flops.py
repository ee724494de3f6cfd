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
