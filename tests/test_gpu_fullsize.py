"""Parity at the full size of the bench workload (n = 102,400: a jittered
320 x 320 grid, tile 512), where the oracle cannot factor the whole matrix:

* Sigma generated on the GPU, 4,000 sampled entries against the oracle's
  Matern evaluated one by one at the same distances (1e-13 + 4u x relative,
  the elementwise bar of the smaller tests), for nu = 1/2 and a general nu,
  in the FP64 layout and in the FP32 mode's mixed layout;
* the IND approximation over the whole field (100 blocks of 1,024 points, the
  batched scheduler) against the oracle's per-block log-likelihoods, 1e-10;
* the FP32-mode evaluation in the bench's launch configuration (FP64 band of
  2 tiles, FP64-accurate updates up to 2 tiles from the diagonal): finite,
  bitwise reproducible, l assembled exactly from its log-det and quadratic
  form, and a refinement step below the guard's 1e-5.
"""
import math

import numpy as np
import pytest

import egs_inputs as ei
import oracle

pytestmark = pytest.mark.gpu

N, B = 102400, 512


@pytest.fixture(scope="module")
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    return m


@pytest.fixture(scope="module")
def field():
    return ei.jittered_grid(N, seed=ei.CONFIG3.seed)


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.3, 0.07, 1.3)])
def test_sampled_sigma_entries(egs, field, theta):
    import torch
    from gpu_util import locs_dev
    T = N // B
    buf = torch.empty(egs.egs_tiles_bytes(N, B) // 8, dtype=torch.float64, device="cuda")
    egs.egs_matern_tiles(locs_dev(field), N, theta, B, buf)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    i = rng.integers(0, N, 4000)
    j = rng.integers(0, N, 4000)
    i, j = np.maximum(i, j), np.minimum(i, j)             # lower triangle
    ti, tj, r, c = i // B, j // B, i % B, j % B
    idx = (ti * (ti + 1) // 2 + tj) * B * B + r * B + c
    got = buf[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    dist = np.hypot(field[0, i] - field[0, j], field[1, i] - field[1, j])
    want = oracle.matern(theta, dist)
    u = 2.0 ** -53
    rtol = 1e-13 + 4 * u * dist / theta[1]                 # as in the elementwise tile test
    assert np.all(np.abs(got - want) <= rtol * np.abs(want) + 1e-290)
    del buf


def test_sampled_mixed_layout_entries(egs, field):
    """The FP32-mode layout at full size (FP64 band of 2 tiles, the off-band
    tiles rounded to float; for nu = 1/2 the off-band values come from the
    double-float evaluation): 4,000 sampled entries within one FP32 rounding
    plus the FP64 element bar of the oracle's value, band entries within the
    FP64 bar."""
    import torch
    from gpu_util import locs_dev
    theta, band = (1.0, 0.1, 0.5), 2
    T = N // B
    nbytes = egs.egs_tiles_bytes(N, B, "fp32", band)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    egs.egs_matern_tiles(locs_dev(field), N, theta, B, buf, "fp32", band)
    torch.cuda.synchronize()
    f64 = buf[: T * band * B * B * 8].view(torch.float64)
    f32 = buf[T * band * B * B * 8:].view(torch.float32)
    rng = np.random.default_rng(23)
    i = rng.integers(0, N, 4000)
    j = rng.integers(0, N, 4000)
    i, j = np.maximum(i, j), np.minimum(i, j)
    j[:1000] = np.maximum(i[:1000] - rng.integers(0, 2 * B, 1000), 0)   # a quarter near the band
    ti, tj, r, c = i // B, j // B, i % B, j % B
    dist = np.hypot(field[0, i] - field[0, j], field[1, i] - field[1, j])
    want = oracle.matern(theta, dist)
    u = 2.0 ** -53
    rtol = 1e-13 + 4 * u * dist / theta[1]
    inb = ti - tj < band
    i64 = (ti * band + (ti - tj)) * B * B + r * B + c
    q = ti - band
    i32 = (q * (q + 1) // 2 + tj) * B * B + r * B + c
    got64 = f64[torch.as_tensor(i64[inb], device="cuda")].cpu().numpy()
    got32 = f32[torch.as_tensor(i32[~inb], device="cuda")].cpu().numpy().astype(np.float64)
    assert inb.sum() > 100 and (~inb).sum() > 1000
    assert np.all(np.abs(got64 - want[inb]) <= rtol[inb] * np.abs(want[inb]) + 1e-290)
    w32 = want[~inb]
    assert np.all(np.abs(got32 - w32) <= (2.0 ** -24 + rtol[~inb]) * np.abs(w32) + 1e-38)
    del buf


def test_ind_over_the_whole_field(egs, field):
    from gpu_util import locs_dev, dev
    theta = (1.0, 0.1, 0.5)
    z = ei.normal(3, N)
    ll, info = egs.egs_loglik_ind(locs_dev(field), dev(z), theta, N, tile=B, super_tiles=2)
    ref = 0.0
    for s in range(0, N, 2 * B):
        ref += oracle.loglik_lapack(field[:, s:s + 2 * B], z[s:s + 2 * B], theta)["loglik"]
    assert abs(ll - ref) <= 1e-10 * abs(ref)


def test_fp32_mode_bench_configuration(egs, field):
    from gpu_util import locs_dev, dev
    theta = (1.0, 0.1, 0.5)
    dl, dz = locs_dev(field), dev(ei.normal(0, N))
    a, ia = egs.egs_loglik_ex(dl, dz, theta, N, "fp32", tile=B, band=2, xband=3)
    b, _ = egs.egs_loglik_ex(dl, dz, theta, N, "fp32", tile=B, band=2, xband=3)
    assert math.isfinite(a) and a == b
    assembled = -0.5 * ia["quad"] - 0.5 * ia["logdet"] - 0.5 * N * math.log(2.0 * math.pi)
    assert abs(a - assembled) <= 1e-12 * abs(a)
    assert abs(ia["quad"] - ia["quad_unrefined"]) <= 1e-5 * abs(ia["quad"])
