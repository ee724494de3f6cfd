"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Element-wise for the covariance tiles, the factor and the solve; scalar for
log|Sigma|, Z^T Sigma^-1 Z and l.  Sizes span several tiles and a ragged tail.
Tolerances:
  * Sigma entries: 1e-13 + 4 x u relative, u = 2^-53, x = r / theta2.  Both
    sides evaluate Eq. 2 to ~1e-15 with different Bessel methods; on top of
    that C(x) decays like e^-x, so a one-ulp difference in how x = r / theta2
    is rounded moves C by x u relative (the conditioning of e^-x);
  * l, log|Sigma|, Z^T Sigma^-1 Z: |d|/|ref| <= 1e-10 in FP64 (the stated
    parity bar), on well-conditioned workloads shaped like the paper's.
"""
import math

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


def _lower_tiles_equal(got, want, rtol, atol=1e-300):
    """rtol is a scalar or a list of per-tile arrays."""
    worst = 0.0
    for t, (g, w) in enumerate(zip(got, want)):
        tol = rtol if np.isscalar(rtol) else rtol[t]
        d = np.abs(g - w) / (np.abs(w) + atol) / tol
        worst = max(worst, float(d.max()))
    assert worst <= 1.0, worst
    return worst


def _x_tiles(locs, theta2, b):
    """x = r / theta2 for every entry, in the lower-tile layout."""
    d = np.hypot(locs[0][:, None] - locs[0][None, :], locs[1][:, None] - locs[1][None, :])
    return oracle.tiles_lower(d / theta2, b)


THETAS = [
    (1.0, 0.1, 0.5),     # exponential (Section 2.2)
    (1.7, 0.08, 1.5),    # closed form 3/2
    (0.6, 0.2, 2.5),     # closed form 5/2
    (1.0, 0.2, 1.3),     # general nu, mu = 0.3, N = 1
    (1.2, 0.05, 0.3),    # general nu, N = 0
    (0.9, 0.15, 0.7),    # mu = -0.3
    (1.0, 0.3, 1.0),     # Whittle (mu = 0)
    (1.0, 0.1, 3.5),     # mu = -1/2 exactly, N = 4
    (2.0, 0.004, 0.9),   # large x (to ~350)
    (1.0, 5.0, 1.9),     # small x only
]


@pytest.mark.parametrize("theta", THETAS)
def test_matern_tiles_elementwise(egs, theta):
    from gpu_util import locs_dev, tiles_to_list
    import torch
    n, b = 700, 128
    T = -(-n // b)
    locs = ei.jittered_grid(n, seed=3)
    S = oracle.cov_matrix(locs, theta)
    want = oracle.tiles_lower(S, b)
    buf = torch.empty(egs.egs_tiles_bytes(n, b) // 8, dtype=torch.float64, device="cuda")
    egs.egs_matern_tiles(locs_dev(locs), n, theta, b, buf)
    torch.cuda.synchronize()
    got = tiles_to_list(buf, T, b)
    u = 2.0 ** -53
    tol = [1e-13 + 4 * u * x for x in _x_tiles(locs, theta[1], b)]
    _lower_tiles_equal(got, want, rtol=tol)


@pytest.mark.parametrize("prec,band,theta", [
    ("fp32", 2, (1.0, 0.1, 1.3)), ("tf32", 3, (1.0, 0.1, 1.3)), ("bf16", 2, (1.0, 0.1, 1.3)),
    # closed-form kinds: the off-band tiles come from the double-float evaluation
    ("fp32", 2, (1.0, 0.1, 0.5)), ("fp32", 3, (1.7, 0.08, 1.5)), ("tf32", 2, (0.6, 0.2, 2.5)),
    ("fp32", 2, (2.0, 0.004, 0.5)),   # x up to ~350: values down to the float range and below
])
def test_matern_tiles_mixed_layout(egs, prec, band, theta):
    """The mixed-precision layout of egs_matern_tiles: band tiles (i - j <
    band) as doubles at i * band + (i - j), the other tiles as floats at
    (i - band)(i - band + 1) / 2 + j of the array that follows; doubles within
    the FP64 element bar of the oracle, floats within one FP32 rounding of the
    oracle's value (plus the same bar, and 1e-38 absolute for values at the
    bottom of the float range)."""
    import torch
    n, b = 1000, 128
    T = -(-n // b)
    locs = ei.jittered_grid(n, seed=3)
    want = oracle.tiles_lower(oracle.cov_matrix(locs, theta), b)
    xs = _x_tiles(locs, theta[1], b)
    nbytes = egs.egs_tiles_bytes(n, b, prec, band)
    n64 = T * band                      # band slots per tile row (the first rows leave some unused)
    assert nbytes == n64 * b * b * 8 + (T - band) * (T - band + 1) // 2 * b * b * 4
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    from gpu_util import locs_dev
    egs.egs_matern_tiles(locs_dev(locs), n, theta, b, buf, prec, band)
    torch.cuda.synchronize()
    raw = buf.cpu().numpy()
    f64 = raw[: n64 * b * b * 8].view(np.float64).reshape(-1, b, b)
    f32 = raw[n64 * b * b * 8:].view(np.float32).reshape(-1, b, b)
    u = 2.0 ** -53
    for i in range(T):
        for j in range(i + 1):
            t = i * (i + 1) // 2 + j
            tol = 1e-13 + 4 * u * xs[t]
            if i - j < band:
                got = f64[i * band + (i - j)]
                assert np.all(np.abs(got - want[t]) <= tol * np.abs(want[t]) + 1e-300), (i, j)
            else:
                r = i - band
                got = f32[r * (r + 1) // 2 + j].astype(np.float64)
                assert np.all(np.abs(got - want[t]) <= (2.0 ** -24 + tol) * np.abs(want[t]) + 1e-38), (i, j)


def _spd_case(n, theta, seed=5):
    locs = ei.jittered_grid(n, seed=seed)
    S = oracle.cov_matrix(locs, theta)
    return locs, S


@pytest.mark.parametrize("n,b", [(700, 128), (1000, 192), (257, 64)])
def test_potrf_tiles_vs_oracle(egs, n, b):
    import scipy.linalg as sla
    from gpu_util import tiles_from_list, tiles_to_list
    theta = (1.0, 0.05, 0.5)
    _, S = _spd_case(n, theta)
    T = -(-n // b)
    buf = tiles_from_list(oracle.tiles_lower(S, b))
    assert egs.egs_potrf_tiles(buf, n, b) == -1
    got = tiles_to_list(buf, T, b)
    Lref = sla.cholesky(S, lower=True)
    want = oracle.tiles_lower(Lref, b)
    # the kernel zeroes the strict upper triangle of diagonal tiles, as L has
    for t, (g, w) in enumerate(zip(got, want)):
        assert np.allclose(g, w, rtol=1e-11, atol=1e-13), t
    # backward error of the factor itself
    P = np.zeros((T * b, T * b))
    idx = 0
    for i in range(T):
        for j in range(i + 1):
            P[i * b:(i + 1) * b, j * b:(j + 1) * b] = got[idx]
            idx += 1
    Lg = P[:n, :n]
    assert np.abs(Lg @ Lg.T - S).max() <= 1e-13 * np.abs(S).max()


def test_trsv_tiles_vs_oracle(egs):
    from gpu_util import dev, tiles_from_list
    import scipy.linalg as sla
    import torch
    n, b = 900, 128
    theta = (1.0, 0.07, 0.5)
    _, S = _spd_case(n, theta, seed=9)
    L = sla.cholesky(S, lower=True)
    z = ei.normal(11, n)
    buf = tiles_from_list(oracle.tiles_lower(L, b))
    zd = dev(z)
    yd = torch.empty_like(zd)
    logdet, quad = egs.egs_trsv_tiles(buf, n, b, zd, yd)
    y = oracle.forward_solve(L, z)
    assert np.allclose(yd.cpu().numpy(), y, rtol=1e-12, atol=1e-12)
    assert abs(logdet - 2 * np.sum(np.log(np.diag(L)))) <= 1e-12 * abs(logdet)
    assert abs(quad - y @ y) <= 1e-12 * abs(quad)


def _loglik_case(n, theta, seed):
    p = ei.Problem(n=n, theta=theta, seed=seed)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    return locs, z


@pytest.mark.parametrize("n,theta,tile,seed", [
    (1600, (1.0, 0.1, 0.5), 320, 0),     # config 1: 40 x 40 grid, tile 320
    (1000, (1.0, 0.15, 1.3), 128, 4),    # general nu
    (777, (2.0, 0.05, 0.8), 64, 7),      # ragged, many tiles
    (1, (1.5, 0.1, 0.5), 64, 2),         # n = 1
    (2, (1.0, 0.2, 1.3), 64, 2),         # n = 2
])
def test_loglik_vs_oracle(egs, n, theta, tile, seed):
    from gpu_util import locs_dev, dev
    locs, z = _loglik_case(n, theta, seed)
    ref = oracle.loglik(locs, z, theta)
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp64", tile=tile)
    assert abs(ll - ref["loglik"]) <= 1e-10 * abs(ref["loglik"]), (ll, ref)
    assert abs(info["logdet"] - ref["logdet"]) <= 1e-10 * max(1.0, abs(ref["logdet"]))
    assert abs(info["quad"] - ref["quad"]) <= 1e-10 * abs(ref["quad"])
    assert info["fail_index"] == -1


def test_loglik_host_pointers_match_device(egs):
    from gpu_util import locs_dev, dev
    n, theta = 1000, (1.0, 0.1, 0.5)
    locs, z = _loglik_case(n, theta, 1)
    a = egs.egs_loglik(locs_dev(locs), dev(z), theta, n)
    b = egs.egs_loglik(np.ascontiguousarray(locs.reshape(-1)), np.ascontiguousarray(z), theta, n)
    assert a == b


def test_loglik_deterministic(egs):
    from gpu_util import locs_dev, dev
    n, theta = 1500, (1.0, 0.2, 1.3)
    locs, z = _loglik_case(n, theta, 2)
    ld, zd = locs_dev(locs), dev(z)
    vals = [egs.egs_loglik(ld, zd, theta, n) for _ in range(3)]
    assert vals[0] == vals[1] == vals[2]


def test_not_positive_definite(egs):
    from gpu_util import locs_dev, dev
    # a very smooth, very long-range field on 600 points: Sigma is singular in FP64
    n, theta = 600, (1.0, 5.0, 4.2)
    locs = ei.jittered_grid(n, seed=1)
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.loglik(locs, np.ones(n), theta)
    with pytest.raises(egs.NotPositiveDefinite):
        egs.egs_loglik_ex(locs_dev(locs), dev(np.ones(n)), theta, n, "fp64", tile=128)
    try:
        egs.egs_loglik_ex(locs_dev(locs), dev(np.ones(n)), theta, n, "fp64", tile=128)
    except egs.NotPositiveDefinite as exc:
        assert "row" in str(exc)


@pytest.mark.parametrize("theta", [(-1.0, 0.1, 0.5), (1.0, 0.0, 0.5), (1.0, 0.1, float("nan")), (1.0, 0.1, float("inf"))])
def test_bad_theta(egs, theta):
    from gpu_util import locs_dev, dev
    locs = ei.jittered_grid(100)
    with pytest.raises(egs.EgsError) as e:
        egs.egs_loglik(locs_dev(locs), dev(np.ones(100)), theta, 100)
    assert e.value.status == egs.EGS_ERR_ARG


def test_bad_sizes(egs):
    from gpu_util import locs_dev, dev
    locs = ei.jittered_grid(100)
    with pytest.raises(egs.EgsError):
        egs.egs_loglik(locs_dev(locs), dev(np.ones(100)), (1, 0.1, 0.5), 0)
    with pytest.raises(egs.EgsError):
        egs.egs_loglik_ex(locs_dev(locs), dev(np.ones(100)), (1, 0.1, 0.5), 100, "fp64", tile=100)


@pytest.mark.parametrize("n,tile", [(900, 128), (1600, 320)])
def test_simulate_matches_oracle(egs, n, tile):
    """Algorithm 1 on the GPU: z = L e against the oracle's L e."""
    from gpu_util import locs_dev, dev
    import torch
    theta = (1.0, 0.1, 0.5)
    p = ei.Problem(n=n, theta=theta, seed=8)
    locs, e = p.locations(), p.e()
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    egs.egs_simulate(locs_dev(locs), dev(e), theta, n, z, tile=tile)
    want = oracle.simulate_z(locs, theta, e)
    got = z.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
