"""Kriging prediction on the GPU (Eq. 5, Algorithm 3) against the oracle.

FP64 bar: |z_gpu - z_oracle| <= 1e-9 max|Z_2| (both solve Sigma_22 X = Z_2 in
FP64 with different factorisation orders, so they agree to about
kappa(Sigma_22) 1e-16); FP32 mixed mode (split-TF32 off-band, FP64-accurate
band updates, one FP64 refinement step): 1e-6 max|Z_2|.  Also the
interpolation property and a hold-out MSE below the field variance.
"""
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


def _split(n_total, theta, seed, m):
    """Simulate Z on n_total jittered-grid points; hold out every
    (n_total // m)-th point as the prediction set."""
    p = ei.Problem(n=n_total, theta=theta, seed=seed)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    step = n_total // m
    held = np.zeros(n_total, bool)
    held[::step] = True
    return locs[:, ~held], z[~held], locs[:, held], z[held]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-6)])
@pytest.mark.parametrize("theta,tile", [((1.0, 0.1, 0.5), 256), ((1.5, 0.05, 1.2), 256)])
def test_predict_matches_oracle(egs, prec, tol, theta, tile):
    import torch
    from gpu_util import locs_dev, dev
    lo, zo, ln, zn = _split(4200, theta, 12, 300)
    n, m = zo.size, zn.size
    ref = oracle.predict(lo, zo, ln, theta)
    out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
    egs.egs_predict(locs_dev(lo), dev(zo), n, locs_dev(ln), m, theta, out, precision=prec, tile=tile)
    got = out.cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(zo))
    mse = float(np.mean((got - zn) ** 2))
    print("%s theta=%s max err %.2e  hold-out MSE %.3e (variance %.2f)" % (prec, theta, err, mse, theta[0]))
    assert err <= tol
    assert mse < 0.5 * theta[0]


def test_predict_interpolates_and_host_io(egs):
    from gpu_util import locs_dev, dev
    theta = (1.0, 0.1, 0.5)
    p = ei.Problem(n=1000, theta=theta, seed=13)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    new = np.ascontiguousarray(locs[:, ::9])
    out = np.empty(new.shape[1])
    egs.egs_predict(np.ascontiguousarray(locs.reshape(-1)), np.ascontiguousarray(z), 1000,
                    np.ascontiguousarray(new.reshape(-1)), new.shape[1], theta, out, tile=128)
    assert np.max(np.abs(out - z[::9])) <= 1e-8 * np.max(np.abs(z))
