#!/usr/bin/env python3
"""Benchmark: exact Gaussian log-likelihood evaluations per second on GB300.

One step = one full evaluation of Eq. 1 by Algorithm 2 (Matern generation,
tile Cholesky, forward solve, log-determinant, quadratic form; in mixed
precision also the FP64 refinement) on the n = 102,400 workload: a jittered
320 x 320 grid over [0, 1]^2, theta = (1, 0.1, 0.5), tile 512.  Default: the
FP32 mixed mode with the stated FP64 band of 2 tiles (FP32 off-band storage,
split-FP16 tensor-core updates of the off-band tiles, FP64-accurate updates of
every tile within 3 of the diagonal: --xband 3); --precision fp32|tf32|bf16,
--band and --xband give the other variants.  Inputs are resident in HBM when
the timed region starts; the tile matrix (up to 42 GB) is regenerated every
step, far larger than L2.

Besides the timed mixed-precision steps, the default line carries the rest of
the metric: one FP64 evaluation of the same inputs ("fp64": evals/s, POTRF
TFLOP/s, the FP64 update's roofline; "mixed_over_fp64", "dl_rel_vs_fp64"),
the serving loop's p50 / p99 at 0.8 of its measured capacity ("serve"), and
the oracle on a bounded host sample ("cpu_baseline").

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|tf32|bf16|fp32]
  python bench.py --impl reference ...   (the CPU oracle as the reference arm)
Under torchrun each rank runs an independent replica (the single
factorisation does not shard); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "loglik evals/s & POTRF TFLOP/s at n=102400 FP64 vs mixed; serve p50/p99 ms"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # SMs x DFMA/clk/SM x flop/FMA x max clock
# k_tc_gemm, split FP16 update: 3.560 GB of DRAM traffic (1.888 read + 1.673 written) for 1.331e12
# executed flop in one launch (ncu; n = 32,768, tile 512, the bulk update of step 2: 1,653 output tiles)
SPLIT_F16_DRAM_BYTES_PER_FLOP = 3.5605e9 / 1.3312e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="egs", choices=["egs", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--n", type=int, default=102400, help="development override; the workload is n=102400")
    ap.add_argument("--tile", type=int, default=512)
    ap.add_argument("--band", type=int, default=2)
    ap.add_argument("--xband", type=int, default=3,
                    help="FP32 mode: tiles with i - j < xband get FP64-accurate updates (those beyond the band stay "
                         "FP32 in storage); 0 = band")
    ap.add_argument("--theta", default="1.0,0.1,0.5")
    ap.add_argument("--e2e-steps", type=int, default=-1, help="steps of the end-to-end leg (default: = steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="config3",
                    choices=["config3", "config2-mle", "config3-mle", "config4-batched", "config5-serve", "generate"],
                    help="config3 (default): one n=102,400 evaluation per step; the others are the "
                         "MLE, batched and serving workloads, and the Matern generation alone")
    ap.add_argument("--nprob", type=int, default=512, help="config4-batched: problems in the batch")
    ap.add_argument("--evals", type=int, default=50, help="config2-mle: likelihood evaluations")
    ap.add_argument("--requests", type=int, default=48, help="config5-serve: requests per arrival rate")
    ap.add_argument("--cpu-sample-n", type=int, default=8192,
                    help="oracle sample size of the reference arm (one sample per step)")
    ap.add_argument("--cpu-baseline-n", type=int, default=16384,
                    help="oracle sample size of the cpu_baseline object of the default line (one sample)")
    ap.add_argument("--no-fp64", action="store_true", help="config3: skip the one FP64 evaluation")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="config3: requests of the serving leg at 0.8 of capacity (0 = skip)")
    ap.add_argument("--trace", default="", help="config3: write the per-launch trace of the untimed breakdown step "
                                                 "to this CSV file")
    return ap.parse_args()


def timeline_summary(trace) -> dict:
    """Per-stream busy time by kernel class over the factorisation, and how
    long the main stream stood idle (waiting for the lookahead chain), from
    egs_trace_last() records (class, step, stream, start_ms, end_ms)."""
    fac = [r for r in trace if r[1] >= 0]
    if not fac:
        return {}
    busy = {"main": {}, "side": {}}
    for cls, _, st, t0, t1 in fac:
        d = busy["main" if st == 0 else "side"]
        d[cls] = d.get(cls, 0.0) + (t1 - t0)
    span = max(r[4] for r in fac) - min(r[3] for r in fac)
    main_busy = sum(busy["main"].values())
    return {"factor_span_ms": span, "main_ms": busy["main"], "side_ms": busy["side"],
            "main_idle_ms": span - main_busy,
            "note": "CUDA events around every launch of one untimed step; main = the call's stream, side = the "
                    "lookahead chain's stream"}


def max_over_ranks(value: float, world: int, device: str) -> float:
    """The largest per-rank value (the slowest replica's time); value itself
    when there is one rank.  Uses the default process group."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Units processed by all replicas over the slowest replica's time."""
    return world * units_per_rank / seconds_max


def workload_name(a) -> str:
    m = int(round(math.sqrt(a.n)))
    grid = "%dx%d jittered grid" % (m, m) if m * m == a.n else "jittered grid"
    extra = ""
    if a.precision == "fp32" and a.xband > a.band:
        extra = " (FP64-accurate updates up to %d tiles from the diagonal)" % (a.xband - 1)
    return "n=%d (%s over [0,1]^2), theta=(%s), tile %d, %s, FP64 band %d%s" % (
        a.n, grid, a.theta, a.tile, a.precision, a.band, extra)


def flop_counts(n: int, b: int) -> dict:
    """Algorithmic flops of the tile Cholesky per kernel class (padded to T*b)."""
    T = -(-n // b)
    potrf = T * b ** 3 / 3.0
    trsm = T * (T - 1) / 2.0 * b ** 3
    syrk = T * (T - 1) / 2.0 * b ** 3
    gemm = sum((T - k - 1) * (T - k - 2) / 2.0 for k in range(T)) * 2.0 * b ** 3
    return {"potrf": potrf, "trsm": trsm, "update": syrk + gemm, "total_n3": n ** 3 / 3.0, "T": T}


def band_band_flops(n: int, b: int, band: int) -> float:
    """FP64 updates whose two operands are band tiles: per step, the first
    (band-1)(band)/2 tiles of the trailing triangle (SYRK b^3, GEMM 2 b^3)."""
    T = -(-n // b)
    tot = 0.0
    for k in range(T - 1):
        nb = min(band - 1, T - k - 1)
        tot += nb * b ** 3 + (nb * (nb - 1) / 2.0) * 2 * b ** 3
    return tot


def band_out_flops(n: int, b: int, band: int, xband: int = 0) -> float:
    """Updates whose output lies within xband (>= band) of the diagonal
    (m - n < xband) but whose operands are not both FP64 band tiles: the
    FP64-accurate slice products of the FP32 mode."""
    T = -(-n // b)
    xband = max(xband, band)
    tot = 0.0
    for k in range(T - 1):
        for c in range(k + 1, T):
            for d in range(xband):
                m = c + d
                if m < T and m - k >= band:
                    tot += b ** 3 if d == 0 else 2 * b ** 3
    return tot


def tensor_peak(precision: str, sustained: bool = False) -> dict:
    """Dense tensor peak for the operand type, from the measured bf16 figure
    (the burst figure for a kernel timed alone, the sustained one for a
    kernel timed inside a long step)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    try:
        with open(path) as f:
            mp = json.load(f)
        bf16 = float(mp[key])
        src = "measured bf16 (MEASURED_PEAKS.json %s, %s)" % (key, "sustained" if sustained else "burst")
    except Exception:
        bf16 = 1700.0 if sustained else 1900.0
        src = "fallback bf16 %s PFLOP/s" % ("1.7 sustained" if sustained else "1.9 burst")
    if precision == "tf32":
        return {"tflops": bf16 * 0.5, "source": src + " x 1/2 (nominal tf32:bf16 dense ratio 1.1:2.25)"}
    if precision == "fp32":
        # the FP32 mode's off-band update runs FP16 MMAs (split FP16); the
        # dense FP16 and BF16 rates are the same
        return {"tflops": bf16, "source": src + " (FP16 products; nominal dense fp16 = bf16 rate)"}
    return {"tflops": bf16, "source": src}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(a, theta, sample_n: int) -> dict:
    """The CPU oracle (as it stands) on one bounded sample of the workload,
    extrapolated per phase to the full n: generation and solve by n^2,
    Cholesky by n^3."""
    import numpy as np
    import scipy.linalg as sla

    import egs_inputs as ei
    import oracle

    locs = ei.jittered_grid(sample_n, seed=0)
    z = ei.normal(0, sample_n)
    t0 = time.perf_counter()
    S = oracle.cov_matrix(locs, theta)
    t1 = time.perf_counter()
    L = sla.cholesky(S, lower=True, overwrite_a=True, check_finite=False)
    t2 = time.perf_counter()
    y = sla.solve_triangular(L, z, lower=True, check_finite=False)
    _ = 2 * np.sum(np.log(np.diag(L))) + y @ y
    t3 = time.perf_counter()
    r = a.n / sample_n
    t_full = (t1 - t0) * r ** 2 + (t2 - t1) * r ** 3 + (t3 - t2) * r ** 2
    cores = len(os.sched_getaffinity(0))
    return {"value": 1.0 / t_full, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": "one oracle evaluation (C Matern + LAPACK dpotrf/dtrsv, FP64) at n=%d on the same "
                      "jittered-grid recipe, %.1f s; extrapolated to n=%d by n^2 (generation %.2f s, solve %.3f s) "
                      "and n^3 (Cholesky %.2f s)" % (sample_n, t3 - t0, a.n, t1 - t0, t3 - t2, t2 - t1),
            "sample_seconds": t3 - t0, "extrapolated_seconds_per_eval": t_full}


def run_reference(a, rank: int):
    if rank != 0:
        return
    theta = tuple(float(v) for v in a.theta.split(","))
    sample_n = min(a.cpu_sample_n, a.n)
    vals = []
    for i in range(a.warmup + a.steps):
        cb = cpu_baseline(a, theta, sample_n)
        if i >= a.warmup:
            vals.append(cb["extrapolated_seconds_per_eval"])
    t = statistics.median(vals)
    v = 1.0 / t
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "n": a.n, "precision": "fp64", "tile": None},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _to_dev(a):
    import numpy as np
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def run_mle(a, egs):
    """Config 2: n = 25,600 (160 x 160), theta = (1, 0.2, 1.3), Z simulated on the
    GPU by Algorithm 1; one MLE run of --evals derivative-free evaluations in
    FP64 and one in --precision, theta-hat compared.  config3-mle: the same
    on the config-3 field (theta = (1, 0.1, 0.5)) at n = 25,600, where an FP64
    fit is affordable (at n = 102,400 one FP64 evaluation takes ~290 s)."""
    import torch
    import egs_inputs as ei
    from paper_1708_02835_gb300 import mle
    p = ei.CONFIG2
    n = p.n if a.n == 102400 else a.n
    theta = p.theta if a.workload == "config2-mle" else ei.CONFIG3.theta
    locs = ei.jittered_grid(n, seed=p.seed)
    dl, de = _to_dev(locs.reshape(-1)), _to_dev(ei.normal(p.seed, n))
    dz = torch.empty(n, dtype=torch.float64, device="cuda")
    egs.egs_simulate(dl, de, theta, n, dz)
    start = (0.5, 0.1, 1.0)
    out = {}
    for prec in (["fp64", a.precision] if a.precision != "fp64" else ["fp64"]):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = mle.fit(dl, dz, n, prec, start=start, max_evals=a.evals, tile=0 if prec == "fp64" else 512,
                    band=0 if prec == "fp64" else a.band, xband=a.xband)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[prec] = {"theta_hat": list(r.theta), "loglik": r.loglik, "evals": r.evals, "seconds": dt,
                     "evals_per_s": r.evals / dt, "fp64_fallbacks": r.fallbacks}
    line = {"metric": "MLE log-likelihood evaluations/s (%s)" % a.workload, "value": out["fp64"]["evals_per_s"],
            "unit": "evals/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "n=%d (160x160 jittered grid), theta=%s, Z by Algorithm 1 on the GPU, "
                                   "bounded Nelder-Mead from %s over [0.01,5]^3" % (n, tuple(theta), start), "n": n,
                       "band": a.band, "xband": a.xband if a.precision == "fp32" else None},
            "runs": out, "theta_true": list(theta)}
    if len(out) > 1:
        f, m = out["fp64"]["theta_hat"], out[a.precision]["theta_hat"]
        line["theta_hat_max_rel_diff"] = max(abs(x - y) / abs(x) for x, y in zip(f, m))
    print(json.dumps(line), flush=True)


def run_batched(a, egs):
    """Config 4: 512 independent problems, n ~ U{256..4096} on random sub-squares,
    own theta each; FP64 and FP32-off-band (EGS_MIX_FP32) batches, each with its
    tile picked by measuring 64 / 128 / 256.  The line's value is the FP64
    batch; the FP32-off-band batch is reported beside it."""
    import numpy as np
    import torch
    import egs_inputs as ei
    probs = ei.batched_problems(a.nprob)
    ns = [p.n for p in probs]
    dl = [_to_dev(p.locations().reshape(-1)) for p in probs]
    dz = [_to_dev(p.e()) for p in probs]
    th = np.array([p.theta for p in probs])
    flops = sum(n ** 3 / 3.0 for n in ns)
    stream = torch.cuda.current_stream()

    def measure(prec):
        # the library's autotuner times tiles 64 / 128 / 256 on these inputs
        # and stores the best for egs_batch(tile=0)
        best, tune = egs.egs_batch_autotune(ns, dl, dz, th, prec)
        B = egs.egs_batch(ns, tile=0, precision=prec)
        assert B.tile == best
        for _ in range(a.warmup):
            out, stat = B.run(dl, dz, th)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            out, stat = B.run(dl, dz, th, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        tfl = flops / (ms / 1e3) / 1e12
        r = {"problems_per_s": len(ns) / (ms / 1e3), "ms_per_batch": ms, "tile": best, "graph_kernels": B.launches,
             "persistent_tasks": B.tasks, "autotune_ms": {str(k): v for k, v in tune.items()},
             "potrf_tflops_equiv": tfl, "failed": int(np.sum(stat != 0)), "workspace_gb": B.workspace_bytes / 1e9}
        if prec == "fp64":
            r["roofline"] = {"bound": "alu", "kernel": "kb_dag (persistent FP64 batch: generation, tile Cholesky, "
                                                       "forward solve)",
                             "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tfl / FP64_PEAK_TFLOPS,
                             "note": "sum of n^3/3 over the problems / batch time; generation and solve time included"}
        B.close()
        return r, out

    r64, out64 = measure("fp64")
    r32, out32 = measure("fp32")
    ok = np.isfinite(out32) & np.isfinite(out64)
    r32["max_rel_diff_vs_fp64"] = float(np.max(np.abs(out32[ok] - out64[ok]) / np.maximum(1.0, np.abs(out64[ok]))))
    line = {"metric": "batched log-likelihood problems/s (config 4)", "value": r64["problems_per_s"],
            "unit": "problems/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": r64["ms_per_batch"],
            "higher_is_better": True, "dtype": "f64", "data": "synthetic (z ~ N(0, I))",
            "config": {"workload": "%d problems, n ~ U{256..4096}, jittered grids on random sub-squares, own theta"
                                   % a.nprob,
                       "tile": r64["tile"], "graph_kernels": r64["graph_kernels"]},
            "autotune_ms": r64["autotune_ms"], "potrf_tflops_equiv": r64["potrf_tflops_equiv"],
            "roofline": r64["roofline"], "persistent_tasks": r64["persistent_tasks"],
            "not_pd": r64["failed"], "fp32_off_band": r32}
    print(json.dumps(line), flush=True)


def run_generate(a, egs):
    """Sigma(theta) alone (Eq. 2; egs_matern_tiles, FP64 lower tiles) on the
    n-point jittered grid: Matern values per second and bytes written, CUDA
    events on the launching stream."""
    import numpy as np
    import torch
    import egs_inputs as ei
    theta = tuple(float(v) for v in a.theta.split(","))
    n, tile = a.n, a.tile
    dl = _to_dev(ei.jittered_grid(n, seed=0).reshape(-1))
    buf = torch.empty(egs.egs_tiles_bytes(n, tile) // 8, dtype=torch.float64, device="cuda")
    for _ in range(a.warmup):
        egs.egs_matern_tiles(dl, n, theta, tile, buf)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        egs.egs_matern_tiles(dl, n, theta, tile, buf)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    T = -(-n // tile)
    vals = T * (T + 1) / 2 * tile * tile
    line = {"metric": "Matern generation values/s", "value": vals / (ms / 1e3), "unit": "values/s", "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "n=%d jittered grid, theta=(%s), tile %d, FP64 lower tiles"
                                                        % (n, a.theta, tile)},
            "bytes_written_gb_s": vals * 8 / (ms / 1e3) / 1e9}
    print(json.dumps(line), flush=True)


def serve_rates(a, egs, rhos, requests: int, burst: int = 16) -> dict:
    """Config 5: 64 resident fields, n log-uniform in [1000, 40000], nu ~ U(0.3, 2);
    capacity from a closed burst, then open-loop Poisson arrivals of theta
    updates at each fraction rho of it, half FP64 and half mixed requests;
    150 GB HBM budget, 8 slots.  Returns capacity and per-rate statistics."""
    import numpy as np
    import egs_inputs as ei
    fields = ei.serving_fields(64)
    rng = np.random.default_rng(0)
    mixed = a.precision if a.precision != "fp64" else "fp32"

    def server():
        srv = egs.egs_server(150 << 30, max_inflight=8, tile=0, band=a.band, fallback_fp64=True, xband=a.xband)
        return srv, [srv.add_field(np.ascontiguousarray(f.locations().reshape(-1)), f.e(), f.n) for f in fields]

    def request(fids, i):
        f = int(rng.integers(len(fields)))
        th = tuple(float(v) * float(np.exp(rng.normal(0, 0.1))) for v in fields[f].theta)
        return fids[f], th, ("fp64" if i % 2 == 0 else mixed)

    srv, fids = server()
    reqs = [request(fids, i) for i in range(burst)]
    t0 = time.perf_counter()
    tickets = [srv.submit(*r) for r in reqs]
    for t in tickets:
        try:
            srv.wait(t)
        except egs.EgsError:
            pass
    cap = len(reqs) / (time.perf_counter() - t0)
    srv.close()
    results = {}
    for rho in rhos:
        srv, fids = server()
        rate = rho * cap
        gaps = rng.exponential(1.0 / rate, requests)
        tickets = []
        t_next = time.perf_counter()
        for i in range(requests):
            t_next += gaps[i]
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(*request(fids, i)))
        for t in tickets:
            try:
                srv.wait(t)
            except egs.EgsError:
                pass
        st = srv.stats()
        results[str(rho)] = {"rate_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                             "mean_ms": st["mean_ms"], "evals_per_s": st["evals_per_s"], "requests": requests,
                             "completed": st["completed"], "failed_not_pd_or_inaccurate": st["failed"],
                             "inflight_peak": st["inflight_peak"], "bytes_peak": st["bytes_peak"],
                             "mixed_rerun_in_fp64": st["fallbacks"]}
        srv.close()
    return {"capacity_per_s": cap, "burst": burst, "mixed": mixed, "rates": results,
            "workload": "64 fields, n log-uniform [1000, 40000], nu ~ U(0.3, 2), Poisson arrivals, 50/50 FP64 and "
                        "%s (band %d, xband %d; a mixed request the accuracy guard rejects is re-run in FP64 by the "
                        "server), 150 GB budget, 8 slots" % (mixed, a.band, a.xband)}


def run_serve(a, egs):
    """Config 5 at 0.5 / 0.8 / 0.95 of measured capacity, --requests each."""
    r = serve_rates(a, egs, (0.5, 0.8, 0.95), a.requests)
    line = {"metric": "serve p50/p99 ms and evals/s (config 5)", "value": r["rates"]["0.8"]["p50_ms"],
            "unit": "ms (p50 at 0.8 of capacity)", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64/f64+" + r["mixed"], "data": "synthetic (z ~ N(0, I))",
            "config": {"workload": r["workload"], "capacity_per_s": r["capacity_per_s"]},
            "rates": r["rates"]}
    print(json.dumps(line), flush=True)


def fp64_leg(a, egs, dlocs, dz, theta, stream) -> dict:
    """One FP64 evaluation of the same workload (same locations, z, tile),
    CUDA-event timed per phase and per kernel class: the FP64 half of the
    metric.  One evaluation takes minutes (n^3/3 = 3.6e14 flop on the FP64
    pipe), so it is timed once, after the mixed-precision legs."""
    import torch
    fc = flop_counts(a.n, a.tile)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(torch.cuda.current_device()))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ll, info = egs.egs_loglik_ex(dlocs, dz, theta, a.n, "fp64", tile=a.tile, timing=2, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    upd = info["ms_update"]
    achieved = fc["update"] / (upd / 1e3) / 1e12 if upd > 0 else 0.0  # one tile: no trailing update
    nlaunch = max(fc["T"] - 1, 1)
    return {"evals_per_s": 1e3 / ms, "ms_per_eval": ms, "loglik": ll, "logdet": info["logdet"], "quad": info["quad"],
            "potrf_tflops": fc["total_n3"] / (info["ms_factor"] / 1e3) / 1e12,
            "phase_ms": {"generate": info["ms_generate"], "factor": info["ms_factor"], "solve": info["ms_solve"]},
            "kernel_class_ms": {k: info["ms_" + k] for k in ("update", "potrf", "trsm", "trsv")},
            "gpu_launches": info["launches"], "clocks": clocks,
            "roofline": {"bound": "alu", "kernel": "k_update_f64 (SYRK/GEMM trailing update, DFMA)",
                         "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe; no FP64 "
                                        "tensor-core path is used)",
                         "launches": nlaunch, "flops_per_launch": fc["update"] / nlaunch,
                         "ms_per_launch": upd / nlaunch},
            "note": "one evaluation, CUDA events on the launching stream, same inputs as the timed mixed steps"}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank)
        return
    if a.workload != "config3":
        import torch
        import paper_1708_02835_gb300 as egs
        torch.cuda.set_device(local)
        egs.load_library()
        {"config2-mle": run_mle, "config3-mle": run_mle, "config4-batched": run_batched,
         "config5-serve": run_serve, "generate": run_generate}[a.workload](a, egs)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import egs_inputs as ei
    import paper_1708_02835_gb300 as egs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    egs.load_library()
    theta = tuple(float(v) for v in a.theta.split(","))
    n, tile = a.n, a.tile
    locs = ei.jittered_grid(n, seed=0)
    z = ei.normal(0, n)
    dlocs = torch.as_tensor(np.ascontiguousarray(locs.reshape(-1))).cuda()
    dz = torch.as_tensor(z).cuda()
    stream = torch.cuda.current_stream()
    ws_bytes = egs.egs_loglik_workspace_bytes(n, tile, a.precision, a.band)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")

    xband = a.xband if a.precision == "fp32" else 0

    def step(timing):
        return egs.egs_loglik_ex(dlocs, dz, theta, n, a.precision, tile=tile, band=a.band, timing=timing,
                                 workspace=ws, stream=stream, xband=xband)

    for _ in range(a.warmup):
        step(0)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(a.steps):
        ll, info = step(1)  # phase events only; per-launch timing runs once below
        infos.append(info)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    # one more (untimed) step with every launch bracketed by events, for the
    # per-kernel-class breakdown and the roofline's kernel time
    _, info2 = step(3)
    trace = egs.egs_trace_last()
    if a.trace and rank == 0:
        with open(a.trace, "w") as f:
            f.write("class,step,stream,start_ms,end_ms\n")
            for cls, k, st, t0, t1 in trace:
                f.write("%s,%d,%d,%.4f,%.4f\n" % (cls, k, st, t0, t1))
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = whole_job_rate(a.steps, world, ms_max / 1e3)

    # end-to-end leg: pinned host inputs through the public C ABI call
    e2e_steps = a.steps if a.e2e_steps < 0 else a.e2e_steps
    hl = torch.as_tensor(np.ascontiguousarray(locs.reshape(-1))).pin_memory()
    hz = torch.as_tensor(z).pin_memory()
    e2e = None
    if e2e_steps > 0:
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            egs.egs_loglik_ex(hl, hz, theta, n, a.precision, tile=tile, band=a.band, workspace=ws, stream=stream,
                              xband=xband)
        barrier()
        te = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": whole_job_rate(e2e_steps, world, te), "unit": "evals/s",
               "h2d_bytes_per_step": int(hl.numel() * 8 + hz.numel() * 8), "d2h_bytes_per_step": 48,
               "steps": e2e_steps}

    # the FP64 half of the metric (one evaluation of the same inputs) and the
    # serving leg (p50 / p99 at 0.8 of capacity); every replica runs them
    del ws
    torch.cuda.empty_cache()
    fp64 = None
    if not a.no_fp64 and a.precision != "fp64":
        fp64 = fp64_leg(a, egs, dlocs, dz, theta, stream)
    torch.cuda.empty_cache()
    serve = None
    if a.serve_requests > 0:
        serve = serve_rates(a, egs, (0.8,), a.serve_requests)
    torch.cuda.empty_cache()

    if rank == 0:
        fc = flop_counts(n, tile)
        ms_step = ms_max / a.steps
        ms_factor = statistics.mean(i["ms_factor"] for i in infos)
        upd_ms = info2["ms_update"]
        launches_update = max(fc["T"] - 1, 1)
        classes = {k: info2["ms_" + k] for k in ("update", "update_f64", "potrf", "trsm", "trsv", "generate")}
        classes["note"] = ("one extra untimed step with CUDA events around every launch; classes on the side "
                           "stream include time spent waiting for SMs")
        if a.precision == "fp64":
            achieved = fc["update"] / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else 0.0
            roof = {"bound": "alu", "kernel": "k_update_f64 (SYRK/GEMM trailing update)", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe, no tensor path)",
                    "launches_per_step": launches_update,
                    "flops_per_launch": fc["update"] / launches_update, "ms_per_launch": upd_ms / launches_update}
        else:
            # tensor-core trailing update: every update except the FP64 band x
            # band tiles (FP32 mode: except every band output, and each
            # update is three TF32 products hi hi' + lo hi' + hi lo')
            f64_flops = band_band_flops(n, tile, a.band)
            tc_flops = fc["update"] - f64_flops
            products = 1
            if a.precision == "fp32":
                bo = band_out_flops(n, tile, a.band, xband)
                tc_flops -= bo
                f64_flops += bo
                products = 3
            upd_s = upd_ms / 1e3 if upd_ms > 0 else float("inf")  # one tile: no trailing update
            executed = products * tc_flops / upd_s / 1e12
            achieved = tc_flops / upd_s / 1e12
            peak = tensor_peak(a.precision, sustained=True)
            peak_burst = tensor_peak(a.precision, sustained=False)
            # DRAM bytes per executed flop of the split-FP16 update from an ncu
            # capture at n = 32,768, scaled to this launch size by its flops
            # (the output tiles' reduce-adds dominate and grow with the flops)
            traffic = SPLIT_F16_DRAM_BYTES_PER_FLOP * products * tc_flops / (2 * launches_update) \
                if a.precision == "fp32" else None
            roof = {"bound": "tensor", "kernel": "k_tc_gemm (tcgen05 trailing update, %s)" % a.precision,
                    "achieved": achieved, "peak": peak["tflops"], "unit": "TFLOP/s", "frac": achieved / peak["tflops"],
                    "traffic": traffic, "traffic_unit": "bytes per launch (ncu capture at n=32768, scaled by flops)",
                    "peak_source": peak["source"] + "; the kernel runs inside a %.1f s step" % (ms_step / 1e3),
                    "launches_per_step": 2 * launches_update,
                    "flops_per_launch": tc_flops / (2 * launches_update),
                    "ms_per_launch": upd_ms / (2 * launches_update),
                    "executed_tflops": executed, "executed_frac": executed / peak["tflops"],
                    "executed_frac_of_burst": executed / peak_burst["tflops"],
                    "products_per_update": products,
                    "note": "achieved = algorithmic flops of the off-band trailing updates (2 b^3 per tile GEMM, the "
                            "n^3/3 convention) over the tcgen05 launches' event time (two launches per step: column "
                            "k+1, then the rest); executed_* count the %d MMA product(s) per update that the kernel "
                            "issues (%s)" % (products, {"fp32": "split FP16: lo hi' + hi lo' + hi hi' of row-scaled "
                                                                "FP16 halves", "tf32": "one TF32 product",
                                                        "bf16": "one BF16 product"}[a.precision])}
            upd64 = info2["ms_update_f64"]
            if upd64 > 0:
                a64 = f64_flops / (upd64 / 1e3) / 1e12
                kern = "k_update_f64 (band x band, DFMA)"
                if a.precision == "fp32":
                    kern += " + k_tc_ozaki (other band outputs, 15 exact BF16 slice products on tcgen05)"
                roof["fp64_accurate_updates"] = {
                    "kernel": kern, "achieved_fp64_equivalent": a64, "fp64_peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "vs_fp64_peak": a64 / FP64_PEAK_TFLOPS, "flops_per_step": f64_flops,
                    "ms_per_step": upd64,
                    "note": "event time summed over the launches on both streams (they overlap other work)"}
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f64+" + a.precision,
                "data": "synthetic: jittered grid locations, z ~ N(0, I) (throughput does not depend on z)",
                "config": {"workload": workload_name(a), "n": n, "tile": tile, "band": a.band,
                           "precision": a.precision, "parallelism": "replicas x%d" % world,
                           "l2": "inputs larger than L2: the %.1f GB tile matrix is regenerated every step"
                                 % (ws_bytes / 1e9)},
                "potrf_tflops": fc["total_n3"] / (ms_factor / 1e3) / 1e12,
                "phase_ms": {"generate": statistics.mean(i["ms_generate"] for i in infos),
                             "factor": ms_factor, "solve": statistics.mean(i["ms_solve"] for i in infos)},
                "kernel_class_ms": classes,
                "timeline": timeline_summary(trace),
                "loglik": infos[-1]["loglik"],
                "roofline": roof, "clocks": clocks,
                "gpu_launches": int(sum(i["launches"] for i in infos)),
                "e2e": e2e}
        if fp64 is not None:
            line["fp64"] = fp64
            line["mixed_over_fp64"] = (value / world) / fp64["evals_per_s"]
            line["dl_rel_vs_fp64"] = abs(infos[-1]["loglik"] - fp64["loglik"]) / abs(fp64["loglik"])
            line["dlogdet_vs_fp64"] = infos[-1]["logdet"] - fp64["logdet"]
        if serve is not None:
            r = serve["rates"]["0.8"]
            line["serve"] = {"p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "evals_per_s": r["evals_per_s"],
                             "capacity_per_s": serve["capacity_per_s"], "rate_per_s": r["rate_per_s"],
                             "requests": r["requests"], "completed": r["completed"],
                             "mixed_rerun_in_fp64": r["mixed_rerun_in_fp64"], "inflight_peak": r["inflight_peak"],
                             "workload": serve["workload"] + "; capacity from a closed burst of %d requests, then "
                                         "Poisson arrivals at 0.8 of it" % serve["burst"]}
        if not a.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(a, theta, min(a.cpu_baseline_n, n))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
