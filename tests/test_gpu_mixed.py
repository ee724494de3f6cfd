"""Mixed precision (FP64 band, FP32 / TF32 / BF16 off-band on tcgen05, one
FP64 refinement step of the quadratic form) against the FP64 CPU oracle.

Stated bars per result (Eq. 1 assembled from the mixed factor's FP64
log-determinant and the refined quadratic form):
  FP32 (split TF32 off-band, every band-tile update in FP64): |dl|/|l| <= 1e-6;
  TF32: |dl|/|l| <= 1e-6 at these sizes (the error grows about linearly with
  n);  BF16: |dl|/|l| <= 5e-5 (BF16 keeps 8 significant bits, so the off-band
  factor carries ~4e-3 relative rounding per entry).
Single-precision off-band tiles cannot factor very smooth, long-range fields
(condition numbers beyond 1/eps_FP32); there the mixed path must report
EGS_ERR_NOT_PD or EGS_ERR_INACCURATE cleanly rather than return a wrong number.
In the FP32 and TF32 modes the refined quadratic form must be closer to the
oracle's than the unrefined one (with BF16 one refinement step need not
contract).
"""
import numpy as np
import pytest

import egs_inputs as ei
import oracle

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "tf32": 1e-6, "bf16": 5e-5}


@pytest.fixture(scope="module")
def egs():
    import paper_1708_02835_gb300 as m
    m.load_library()
    return m


def _case(n, theta, seed):
    p = ei.Problem(n=n, theta=theta, seed=seed)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    return locs, z, oracle.loglik_lapack(locs, z, theta)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("n,theta,tile,band", [
    (4096, (1.0, 0.1, 0.5), 256, 2),
    (3000, (1.0, 0.05, 0.8), 256, 2),    # ragged tail, general nu
    (4600, (1.5, 0.05, 0.6), 512, 2),    # tile 512 as at n = 102,400
    (4096, (1.0, 0.1, 0.5), 256, 3),     # wider FP64 band
])
def test_mixed_loglik_vs_oracle(egs, prec, n, theta, tile, band):
    from gpu_util import locs_dev, dev
    locs, z, ref = _case(n, theta, 3)
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=tile, band=band)
    rel = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    print("%s n=%d rel l %.2e  logdet %.3e  quad %.2e (unrefined %.2e)" % (
        prec, n, rel, info["logdet"] - ref["logdet"], abs(info["quad"] - ref["quad"]) / ref["quad"],
        abs(info["quad_unrefined"] - ref["quad"]) / ref["quad"]))
    assert info["band"] == band and info["refine_steps"] == 1
    assert rel <= TOL[prec], rel
    if prec != "bf16":
        # one FP64 refinement step contracts when kappa * eps(factor) < 1; the
        # BF16 factor is too inexact for that to hold on these fields
        assert abs(info["quad"] - ref["quad"]) <= abs(info["quad_unrefined"] - ref["quad"]) + 1e-12 * ref["quad"]


def test_mixed_smooth_field_reports_not_pd(egs):
    from gpu_util import locs_dev, dev
    n, theta = 3000, (1.0, 0.15, 1.3)
    locs, z, ref = _case(n, theta, 3)
    ll, _ = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp64", tile=256)
    assert abs(ll - ref["loglik"]) <= 1e-10 * abs(ref["loglik"])
    with pytest.raises(egs.NotPositiveDefinite):
        egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "tf32", tile=256)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_mixed_deterministic(egs, prec):
    from gpu_util import locs_dev, dev
    n, theta = 3000, (1.0, 0.1, 0.5)
    locs, z, _ = _case(n, theta, 5)
    a = [egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=256)[0] for _ in range(3)]
    assert a[0] == a[1] == a[2]


def test_fp32_mode_tracks_fp64_at_n16384(egs):
    """FP32 mode against the FP64 GPU path (itself pinned to the oracle at
    1e-10 by the parity tests) at n = 16,384, tile 512, band 2: 32 tiles per
    side, so the off-band tensor-core work and the FP64 band-output updates
    both run over many steps."""
    from gpu_util import locs_dev, dev
    n, theta = 16384, (1.0, 0.1, 0.5)
    p = ei.Problem(n=n, theta=theta, seed=11)
    locs = p.locations()
    dl = locs_dev(locs)
    e = dev(p.e())
    import torch
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    egs.egs_simulate(dl, e, theta, n, z, tile=512)
    ll64, i64 = egs.egs_loglik_ex(dl, z, theta, n, "fp64", tile=512)
    ll32, i32 = egs.egs_loglik_ex(dl, z, theta, n, "fp32", tile=512, band=2)
    rel = abs(ll32 - ll64) / abs(ll64)
    print("fp32 n=16384 rel l %.2e  dlogdet %.3e" % (rel, i32["logdet"] - i64["logdet"]))
    assert rel <= TOL["fp32"], rel


def test_mixed_small_n_falls_back_to_fp64(egs):
    from gpu_util import locs_dev, dev
    n, theta = 400, (1.0, 0.1, 0.5)
    locs, z, ref = _case(n, theta, 1)
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "tf32", tile=256)
    assert abs(ll - ref["loglik"]) <= 1e-10 * abs(ref["loglik"])


def test_mixed_tile_must_be_multiple_of_256(egs):
    from gpu_util import locs_dev, dev
    locs = ei.jittered_grid(1000)
    with pytest.raises(egs.EgsError):
        egs.egs_loglik_ex(locs_dev(locs), dev(np.ones(1000)), (1, 0.1, 0.5), 1000, "tf32", tile=320)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
@pytest.mark.parametrize("theta", [(1.0, 0.15, 1.3), (1.0, 0.3, 1.0), (1.0, 0.5, 0.5), (2.0, 0.05, 2.0)])
def test_mixed_never_returns_a_gross_error(egs, prec, theta):
    """Smooth or long-range fields push Sigma's condition number towards
    1/eps of the off-band precision.  The mixed path must then either fail
    cleanly (EGS_ERR_NOT_PD, or EGS_ERR_INACCURATE when the FP64 refinement
    step is too large) or return a value close to the oracle's: within 5e-5
    in the FP32 mode (its guard passes only refinement steps below 1e-5,
    measured to keep l within ~2.5e-5), within 1e-3 in TF32 (gross errors
    only)."""
    from gpu_util import locs_dev, dev
    n = 3000
    locs, z, ref = _case(n, theta, 4)
    try:
        ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, prec, tile=256)
    except (egs.NotPositiveDefinite, egs.MixedInaccurate) as e:
        print("%s theta=%s: %s" % (prec, theta, type(e).__name__))
        return
    rel = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    print("%s theta=%s: rel l %.2e" % (prec, theta, rel))
    assert rel <= (5e-5 if prec == "fp32" else 1e-3), rel


@pytest.mark.parametrize("n,theta,tile", [(4096, (1.0, 0.1, 0.5), 256), (4600, (1.5, 0.05, 0.6), 512)])
def test_fp32_mode_extended_band(egs, n, theta, tile):
    """FP64 band of 2 tiles with FP64-accurate (slice-product) updates of the
    tiles one further from the diagonal (xband = 3), which stay FP32 in
    storage: l within the FP32-mode bar of the oracle, and not worse than the
    plain band-2 evaluation by more than rounding."""
    from gpu_util import locs_dev, dev
    locs, z, ref = _case(n, theta, 3)
    l2, _ = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp32", tile=tile, band=2)
    lx, ix = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp32", tile=tile, band=2, xband=3)
    r2 = abs(l2 - ref["loglik"]) / abs(ref["loglik"])
    rx = abs(lx - ref["loglik"]) / abs(ref["loglik"])
    print("fp32 n=%d band 2: rel l %.2e; band 2 + xband 3: %.2e" % (n, r2, rx))
    assert ix["band"] == 2
    assert rx <= TOL["fp32"], rx
    assert rx <= 2 * r2 + 1e-12


def test_fp32_mode_extended_band_tracks_fp64_at_n16384(egs):
    """As test_fp32_mode_tracks_fp64_at_n16384 with xband = 3 (band 2 storage)."""
    from gpu_util import locs_dev, dev
    import torch
    n, theta = 16384, (1.0, 0.1, 0.5)
    p = ei.Problem(n=n, theta=theta, seed=11)
    locs = p.locations()
    dl = locs_dev(locs)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    egs.egs_simulate(dl, dev(p.e()), theta, n, z, tile=512)
    ll64, i64 = egs.egs_loglik_ex(dl, z, theta, n, "fp64", tile=512)
    llx, ix = egs.egs_loglik_ex(dl, z, theta, n, "fp32", tile=512, band=2, xband=3)
    rel = abs(llx - ll64) / abs(ll64)
    print("fp32 n=16384 band 2 + xband 3: rel l %.2e  dlogdet %.3e" % (rel, ix["logdet"] - i64["logdet"]))
    assert rel <= TOL["fp32"], rel


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.05, 0.8)])
def test_refinement_converges_to_the_fp64_quadratic_form(egs, theta):
    """More FP64 refinement steps drive the quadratic form to the accuracy of
    the residual r = Z - Sigma x, whose entries are regenerated tile by tile in
    double-float arithmetic (the closed form at nu = 1/2, the local
    polynomials at nu = 0.8): after four steps Z^T Sigma^-1 Z is within 1e-10
    of the oracle's, and not worse than after one."""
    from gpu_util import locs_dev, dev
    n = 4096
    locs, z, ref = _case(n, theta, 3)
    q = {}
    for steps in (1, 4):
        ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp32", tile=256, band=2, refine=steps)
        assert info["refine_steps"] == steps
        q[steps] = abs(info["quad"] - ref["quad"]) / ref["quad"]
    print("theta %s: quad rel. error after 1 step %.2e, after 4 steps %.2e" % (theta, q[1], q[4]))
    assert q[4] <= 1e-10, q
    assert q[4] <= q[1]


def test_fp32_mode_with_theta1_outside_the_float_pair_range(egs):
    """theta1 = 1e-20 (below the 2^-60 the double-float generator accepts):
    the FP32 tiles and the refinement residual come from the direct FP64
    evaluation, and l, which the scale changes only by known terms, stays
    within the FP32-mode bar of the oracle."""
    from gpu_util import locs_dev, dev
    n, theta = 3000, (1e-20, 0.05, 0.5)
    p = ei.Problem(n=n, theta=theta, seed=9)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    ref = oracle.loglik_lapack(locs, z, theta)
    ll, info = egs.egs_loglik_ex(locs_dev(locs), dev(z), theta, n, "fp32", tile=256, band=2)
    rel = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    print("theta1 1e-20 fp32: rel l %.2e" % rel)
    assert rel <= TOL["fp32"], rel


def test_xband_below_band_is_rejected(egs):
    from gpu_util import locs_dev, dev
    locs = ei.jittered_grid(1000)
    with pytest.raises(egs.EgsError) as e:
        egs.egs_loglik_ex(locs_dev(locs), dev(np.ones(1000)), (1, 0.1, 0.5), 1000, "fp32", tile=256, band=3, xband=2)
    assert e.value.status == egs.EGS_ERR_ARG
