"""Maximum-likelihood driver (Section 6.3): maximise l(theta) of Eq. 1 over
bounded theta with a derivative-free optimiser; every evaluation is one call
of the library's GPU log-likelihood.

The paper drives BOBYQA through NLopt.  NLopt is not part of this stack, so
the driver uses its own bounded Nelder-Mead simplex (Nelder & Mead, Computer
Journal 7, 1965) on u = log(theta), with the bounds enforced by projection
onto the box.  An evaluation whose covariance is not positive definite counts
as l = -inf.  With a mixed precision, a theta whose mixed factorisation fails
(EGS_ERR_NOT_PD) or is flagged too inexact by its refinement step
(EGS_ERR_INACCURATE) is re-evaluated in FP64 (fallback_fp64, on by default),
so that the optimiser never follows a mixed-precision artefact.  Every evaluation is appended to an optional JSONL trace; a run
given an existing trace replays its recorded values instead of re-evaluating,
so an interrupted fit resumes where it stopped.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np


@dataclass
class FitResult:
    theta: tuple
    loglik: float
    evals: int
    history: list = field(default_factory=list)  # (theta, loglik) per evaluation
    fallbacks: int = 0  # mixed-precision evaluations redone in FP64


class _Objective:
    """-l(theta) with a budget, a cache of the trace and NOT_PD -> +inf."""

    def __init__(self, f, max_evals, trace_path=None):
        self.f = f
        self.max_evals = max_evals
        self.history = []
        self.trace_path = trace_path
        self.replay = []
        if trace_path and os.path.exists(trace_path):
            with open(trace_path) as fh:
                for line in fh:
                    line = line.strip()
                    if line:
                        rec = json.loads(line)
                        self.replay.append((tuple(rec["theta"]), rec["loglik"]))

    def __call__(self, theta):
        theta = tuple(float(v) for v in theta)
        idx = len(self.history)
        if idx < len(self.replay) and np.allclose(self.replay[idx][0], theta, rtol=0, atol=0):
            ll = self.replay[idx][1]
        else:
            ll = self.f(theta)
            if self.trace_path:
                with open(self.trace_path, "a") as fh:
                    fh.write(json.dumps({"eval": idx, "theta": list(theta), "loglik": ll}) + "\n")
        ll = float(ll) if ll is not None and math.isfinite(ll) else -math.inf
        self.history.append((theta, ll))
        return -ll

    @property
    def exhausted(self):
        return len(self.history) >= self.max_evals


def nelder_mead_bounded(f, x0, lower, upper, max_evals=50, step=0.5, trace_path=None) -> FitResult:
    """Minimise -l over log(theta) within [log lower, log upper]; f(theta) returns l."""
    lo, hi = np.log(np.asarray(lower, float)), np.log(np.asarray(upper, float))
    obj = _Objective(f, max_evals, trace_path)

    def proj(u):
        return np.minimum(np.maximum(u, lo), hi)

    def val(u):
        return obj(np.exp(proj(u)))

    d = len(x0)
    u0 = proj(np.log(np.asarray(x0, float)))
    simplex = [u0]
    for i in range(d):
        u = u0.copy()
        u[i] = u[i] + step if u[i] + step <= hi[i] else u[i] - step
        simplex.append(proj(u))
    fs = []
    for u in simplex:
        if obj.exhausted:
            break
        fs.append(val(u))
    simplex = simplex[:len(fs)]
    alpha, gamma, rho, sigma = 1.0, 2.0, 0.5, 0.5
    while not obj.exhausted and len(fs) == d + 1:
        order = np.argsort(fs, kind="stable")
        simplex = [simplex[i] for i in order]
        fs = [fs[i] for i in order]
        centroid = np.mean(simplex[:-1], axis=0)
        ur = proj(centroid + alpha * (centroid - simplex[-1]))
        fr = val(ur)
        if fs[0] <= fr < fs[-2]:
            simplex[-1], fs[-1] = ur, fr
            continue
        if fr < fs[0]:
            if obj.exhausted:
                simplex[-1], fs[-1] = ur, fr
                break
            ue = proj(centroid + gamma * (ur - centroid))
            fe = val(ue)
            simplex[-1], fs[-1] = (ue, fe) if fe < fr else (ur, fr)
            continue
        if obj.exhausted:
            break
        uc = proj(centroid + rho * (simplex[-1] - centroid))
        fc = val(uc)
        if fc < fs[-1]:
            simplex[-1], fs[-1] = uc, fc
            continue
        for i in range(1, d + 1):
            if obj.exhausted:
                break
            simplex[i] = proj(simplex[0] + sigma * (simplex[i] - simplex[0]))
            fs[i] = val(simplex[i])
    best = max(obj.history, key=lambda t: t[1])
    return FitResult(theta=best[0], loglik=best[1], evals=len(obj.history), history=list(obj.history))


def fit(locs, z, n: int, precision="fp64", start=(0.5, 0.05, 0.5), lower=(0.01, 0.01, 0.01),
        upper=(5.0, 5.0, 5.0), max_evals: int = 50, tile: int = 0, band: int = 0, trace_path=None,
        stream=None, fallback_fp64: bool = True, xband: int = 0) -> FitResult:
    """Maximum-likelihood estimate of theta with every l(theta) evaluated on the GPU.

    locs (2n doubles, x then y) and z (n doubles) should be device tensors so
    they stay resident across evaluations."""
    from . import binding as egs

    fallbacks = []

    def fp64(theta):
        try:
            return egs.egs_loglik_ex(locs, z, theta, n, "fp64", stream=stream)[0]
        except egs.NotPositiveDefinite:
            return -math.inf

    def loglik(theta):
        try:
            ll, _ = egs.egs_loglik_ex(locs, z, theta, n, precision, tile=tile, band=band, stream=stream,
                                      xband=xband if precision == "fp32" else 0)
            return ll
        except (egs.NotPositiveDefinite, egs.MixedInaccurate):
            if precision == "fp64" or not fallback_fp64:
                return -math.inf
            fallbacks.append(tuple(theta))
            return fp64(theta)

    r = nelder_mead_bounded(loglik, start, lower, upper, max_evals=max_evals, trace_path=trace_path)
    r.fallbacks = len(fallbacks)
    return r
