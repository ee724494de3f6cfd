"""FP64 parity at n = 25,600 with tile 512, the sizes where the FP64 path takes
the kernel variants it uses at full scale (the 64-row panel TRSM, selected
while at least 38 tile rows remain below the diagonal, i.e. steps k <= 11 of
50, and the 64 x 64 FP64 update blocks):

* the tile Cholesky (Algorithm 2, dpotrf; Section 5.2) element by element
  against LAPACK's dpotrf of the same matrix, plus sampled entries of L L^T
  against Sigma (backward error);
* the 160 x 160 jittered-grid workload at theta = (1, 0.2, 1.3), the general-nu
  Bessel path: l, log|Sigma| and Z^T Sigma^-1 Z against the FP64 oracle
  (Eq. 1 by Algorithm 2, Z by Algorithm 1 from the oracle's own factor) at
  |d|/|ref| <= 1e-10.

The oracle work (about 3.3e8 Matern values and one 25,600 LAPACK Cholesky) takes
a minute or two on the host cores.
"""
import numpy as np
import pytest

import egs_inputs as ei
import oracle

pytestmark = pytest.mark.gpu

N, B = 25600, 512


@pytest.fixture(scope="module")
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    return m


def _tiles_of(S, b):
    """Lower tiles of the padded matrix in the library's layout, as one array."""
    n = S.shape[0]
    T = -(-n // b)
    out = np.zeros((T * (T + 1) // 2, b, b))
    t = 0
    for i in range(T):
        for j in range(i + 1):
            blk = S[i * b:(i + 1) * b, j * b:(j + 1) * b]
            out[t, :blk.shape[0], :blk.shape[1]] = blk
            if i == j:
                for r in range(blk.shape[0], b):
                    out[t, r, r] = 1.0
            t += 1
    return out


def test_potrf_tiles_elementwise_n25600_tile512(egs):
    """dpotrf of an exponential covariance (theta2 = 0.1 on the 160 x 160
    grid): |L_gpu - L_lapack| <= 1e-12 max|L| + 1e-10 |L_lapack| for every
    entry (a tiled and a LAPACK Cholesky differ by rounding order only: about
    1e-15 absolute measured on the CPU at n = 8,192), and (L L^T)_ij against
    Sigma_ij at 4,000 sampled entries within 1e-13."""
    import scipy.linalg as sla
    import torch
    locs = ei.jittered_grid(N, seed=21)
    S = np.hypot(locs[0][:, None] - locs[0][None, :], locs[1][:, None] - locs[1][None, :])
    np.exp(-S / 0.1, out=S)
    buf = torch.as_tensor(_tiles_of(S, B).reshape(-1)).cuda()
    assert egs.egs_potrf_tiles(buf, N, B) == -1
    got = buf.cpu().numpy().reshape(-1, B, B)
    del buf
    rng = np.random.default_rng(5)
    i = rng.integers(0, N, 4000)
    j = rng.integers(0, N, 4000)
    want_s = S[i, j].copy()
    L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    del S
    Lmax = np.abs(L).max()
    T = N // B
    worst = 0.0
    t = 0
    for ti in range(T):
        for tj in range(ti + 1):
            w = L[ti * B:(ti + 1) * B, tj * B:(tj + 1) * B]
            g = got[t]
            if ti == tj:
                w = np.tril(w)
            d = np.abs(g - w) / (1e-12 * Lmax + 1e-10 * np.abs(w))
            worst = max(worst, float(d.max()))
            t += 1
    assert worst <= 1.0, worst
    # backward error at sampled entries, from the GPU factor's rows
    def row(r):
        ti = r // B
        out = np.empty(N)
        for tj in range(T):
            if tj <= ti:
                out[tj * B:(tj + 1) * B] = got[ti * (ti + 1) // 2 + tj][r % B]
            else:
                out[tj * B:(tj + 1) * B] = 0.0
        return out
    for a, c, s in zip(i[:400], j[:400], want_s[:400]):
        assert abs(row(a) @ row(c) - s) <= 1e-13, (a, c)


def test_config2_fp64_loglik_vs_oracle(egs):
    """Config 2's field (n = 25,600 on a 160 x 160 jittered grid, seed 0) at
    theta = (1, 0.2, 1.3), tile 512, FP64."""
    from gpu_util import locs_dev, dev
    theta = ei.CONFIG2.theta
    assert tuple(theta) == (1.0, 0.2, 1.3) and ei.CONFIG2.n == N
    p = ei.Problem(n=N, theta=theta, seed=ei.CONFIG2.seed)
    locs = p.locations()
    ref = oracle.simulate_loglik(locs, theta, p.e())
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(ref["z"]), theta, N, "fp64", tile=B)
    print("config 2 FP64: rel l %.2e  logdet %.2e  quad %.2e" % (
        abs(ll - ref["loglik"]) / abs(ref["loglik"]), abs(info["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
        abs(info["quad"] - ref["quad"]) / ref["quad"]))
    assert info["tile"] == B and info["fail_index"] == -1
    assert abs(ll - ref["loglik"]) <= 1e-10 * abs(ref["loglik"])
    assert abs(info["logdet"] - ref["logdet"]) <= 1e-10 * abs(ref["logdet"])
    assert abs(info["quad"] - ref["quad"]) <= 1e-10 * abs(ref["quad"])
