"""The MLE driver's bounded Nelder-Mead (host logic, CPU) and one GPU fit.

Section 6.3: theta-hat maximises Eq. 1 under bounds; the paper uses BOBYQA,
this driver a bounded simplex in log(theta) (same role: derivative-free,
bound-constrained).
"""
import math
import os

import numpy as np
import pytest

from paper_1708_02835_gb300.mle import nelder_mead_bounded


def _bowl(opt):
    lo = np.log(opt)

    def f(theta):
        u = np.log(theta)
        return -float(np.sum((u - lo) ** 2 * np.array([1.0, 3.0, 0.5])))
    return f


def test_converges_inside_bounds():
    opt = (1.3, 0.07, 0.8)
    r = nelder_mead_bounded(_bowl(opt), (0.5, 0.5, 0.5), (0.01,) * 3, (5.0,) * 3, max_evals=300)
    assert r.evals <= 300
    assert np.allclose(r.theta, opt, rtol=2e-3)


def test_bounds_respected_and_budget_exact():
    seen = []

    def f(theta):
        seen.append(theta)
        return -float(np.sum(np.log(theta) ** 2))
    lower, upper = (0.2, 0.3, 0.4), (0.9, 0.8, 0.7)
    r = nelder_mead_bounded(f, (0.5, 0.5, 0.5), lower, upper, max_evals=50)
    assert r.evals == 50 == len(seen)
    for th in seen:
        assert all(l - 1e-12 <= t <= u + 1e-12 for t, l, u in zip(th, lower, upper))
    # the optimum of this bowl lies on the upper bounds (log 1 = 0 outside the box)
    assert np.allclose(r.theta, upper, rtol=1e-2)


def test_not_positive_definite_counts_as_minus_infinity():
    def f(theta):
        if theta[2] > 1.0:
            return -math.inf
        return -float((math.log(theta[2]) - math.log(0.9)) ** 2 + math.log(theta[0]) ** 2 + math.log(theta[1]) ** 2)
    r = nelder_mead_bounded(f, (0.5, 0.5, 0.5), (0.01,) * 3, (5.0,) * 3, max_evals=120)
    assert r.theta[2] <= 1.0 and math.isfinite(r.loglik)


def test_resume_from_trace(tmp_path):
    trace = os.path.join(tmp_path, "trace.jsonl")
    calls = []
    base = _bowl((1.1, 0.2, 0.6))

    def f(theta):
        calls.append(theta)
        return base(theta)
    r1 = nelder_mead_bounded(f, (0.5, 0.5, 0.5), (0.01,) * 3, (5.0,) * 3, max_evals=20, trace_path=trace)
    assert len(calls) == 20
    calls.clear()
    r2 = nelder_mead_bounded(f, (0.5, 0.5, 0.5), (0.01,) * 3, (5.0,) * 3, max_evals=40, trace_path=trace)
    assert len(calls) == 20          # the first 20 come from the trace
    fresh = nelder_mead_bounded(base, (0.5, 0.5, 0.5), (0.01,) * 3, (5.0,) * 3, max_evals=40)
    assert r2.theta == fresh.theta and r2.loglik == fresh.loglik
    assert r1.loglik <= r2.loglik


@pytest.mark.gpu
def test_gpu_fit_fp64_and_mixed():
    import torch
    import egs_inputs as ei
    import oracle
    from paper_1708_02835_gb300 import mle
    theta = (1.0, 0.1, 0.5)
    p = ei.Problem(n=1024, theta=theta, seed=11)
    locs = p.locations()
    z = oracle.simulate_z(locs, theta, p.e())
    dl = torch.as_tensor(np.ascontiguousarray(locs.reshape(-1))).cuda()
    dz = torch.as_tensor(z).cuda()
    start = (0.5, 0.05, 0.5)
    r64 = mle.fit(dl, dz, 1024, "fp64", start=start, max_evals=50, tile=256)
    ll_start = oracle.loglik(locs, z, start)["loglik"]
    assert r64.evals == 50 and r64.loglik >= ll_start
    # the reported maximum is the oracle's value at theta-hat
    assert abs(oracle.loglik(locs, z, r64.theta)["loglik"] - r64.loglik) <= 1e-10 * abs(r64.loglik)
    r32 = mle.fit(dl, dz, 1024, "tf32", start=start, max_evals=50, tile=256, band=2)
    rel = max(abs(a - b) / abs(b) for a, b in zip(r32.theta, r64.theta))
    print("theta64", r64.theta, "theta_tf32", r32.theta, "max rel diff %.2e" % rel)
    assert rel <= 1e-3
