#!/usr/bin/env python3
"""Benchmark of the exact 2D LMS line estimator on the GB300.

Workload (one "step"): one exact LMS fit of n = 8192 int16 points on a line
of random slope angle U(-1.4, 1.4) and integer intercept, inlier noise
U{-3..3}, 45% uniform outliers (the learned-proposal workload), over all
n(n-1)/2 = 33,550,336 candidate slopes, through the C ABI.  Three arms on the
same instances, bit-identical to each other (and, in the tests, to the
oracle):

* ``learned``       (headline ``value``) lms_fit_learned: the set network
                    predicts the slope, branch-and-bound takes its upper bound
                    there, drops slope intervals whose lower bound exceeds it,
                    and sweeps the rest exactly;
* ``quantile_bnb``  lms_fit_bnb without a network: the same branch-and-bound
                    seeded at quantiles of sampled pair slopes;
* ``plain``         lms_fit with the kinetic sweep over every candidate slope.

The previous fixed-slope workload (slope 0.7, 40% outliers) is timed beside
them (``line_40pct``).  Every step uses a fresh seeded instance already
resident in HBM; L2 is flushed (256 MB write) before each step, outside the
timed events.  The two branch-and-bound arms are timed as CUDA-graph
replays, one graph per step captured after the warm-up; the others as
direct calls.  ``e2e`` runs the learned fit through the host-buffer entry
point lms_fit_learned_host, copies included.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank fits its own
instances (weak scaling, no collective on the data path).
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
sys.path.insert(0, ROOT)

N_POINTS = 8192
OUTLIER_FRAC = 0.45
PHI_MAX = 1.4
METRIC = "exact LMS solves/sec at n=8192, learned-seeded branch-and-bound (quantile-seeded and plain sweep alongside)"
UNIT = "solves/s"
WORKLOAD = "single exact LMS fit, n=8192 int16, random slope angle U(-1.4,1.4), 45% outliers (sloped)"
# Algorithmic work of the sweep kernel per event (one pair of points meeting):
# 2 position reads, 4 order/position writes, 3 projections (2 IMAD each),
# 2 window widths and centres, 2 exact candidate comparisons, decode.
SWEEP_INT_OPS_PER_EVENT = 50


def rank_seeds(rank: int, count: int):
    """Instance seeds of one rank: every rank fits its own instances (weak
    scaling, no collective on the data path)."""
    return [rank * 100003 + 1 + s for s in range(count)]


def max_over_ranks(v: float, device=None) -> float:
    """The largest of every rank's value (the slowest rank's time), or v on
    one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the solves of all ranks over the slowest rank's time."""
    return world * steps_per_rank / (max_ms / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _reference_arm(args):
    """The CPU oracle (O2 exact sweep) timed on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1510_01041_gb300 import datagen
    oracle.build()
    cores = oracle.max_threads()
    inst = _instances([1000 + s for s in range(args.warmup + args.steps)])
    for s in range(args.warmup):
        oracle.lms_i16(*inst[s], 0, "sweep")
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.lms_i16(*inst[args.warmup + s], 0, "sweep")
    dt = time.perf_counter() - t0
    v = args.steps / dt
    slopes = N_POINTS * (N_POINTS - 1) // 2
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128",
        "data": "synthetic", "candidate_slopes_per_sec": v * slopes,
        "config": {"workload": WORKLOAD, "n": N_POINTS, "h": N_POINTS // 2 + 1,
                   "algorithm": "CPU oracle O2 (exact rational sweep)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full solves at n={N_POINTS}"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _cpu_baseline(x, y):
    """Bounded oracle sample: one O2 solve of a step's instance (~10 s of CPU work)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.lms_i16(x, y, 0, "sweep")
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"1 full O2 solve at n={N_POINTS} ({dt:.1f} s)"}, r


def _batched(args):
    """4096 sets, n log-uniform in [64, 4096], outlier fraction U(0, 0.45), slope
    angle U(-1.5, 1.5): one batch plan (autotuned) captured into a CUDA graph;
    each step replays the graph on a fresh batch already in HBM."""
    import numpy as np
    import torch

    from paper_1510_01041_gb300 import autotune, build, datagen, lms
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    total = args.warmup + args.steps
    batches = [datagen.batch(4096, 5000 + rank * 1000 + s) for s in range(min(total, 3))]
    x0, y0, off = batches[0]
    xt = torch.from_numpy(x0).to(dev)
    yt = torch.from_numpy(y0).to(dev)
    ot = torch.from_numpy(off).to(dev)
    plan, cfg = autotune.tuned_plan(off, xt, yt, ot)
    out = torch.empty((4096, lms.RESULT_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    plan.fit(xt, yt, ot, out=out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(xt, yt, ot, out=out, stream=s)
    # the sets keep their sizes; their coordinates change between steps
    ys = [torch.from_numpy(b[1][:x0.size] if b[1].size >= x0.size else y0).to(dev) for b in batches]
    for k in range(args.warmup):
        yt.copy_(ys[k % len(ys)])
        g.replay()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    evs = []
    for k in range(args.steps):
        yt.copy_(ys[k % len(ys)])
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b2.record()
        evs.append((a, b2))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b2) for a, b2 in evs)
    res = lms.decode(out)
    assert all(r["status"] in (lms.LMS_OK, lms.LMS_ERR_VERTICAL) for r in res)
    sizes = np.diff(off)
    slopes = int(np.sum(sizes * (sizes - 1) // 2))
    v = 4096 * args.steps / (ms / 1000.0)
    print(json.dumps({
        "metric": "exact LMS solves/sec, batch of 4096 uneven sets", "value": v, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "candidate_slopes_per_sec": v / 4096 * slopes,
        "config": {"workload": "4096 sets, n log-uniform [64,4096], outliers U(0,0.45), angle U(-1.5,1.5)",
                   "autotuned": cfg, "graph": "one CUDA graph per batch", "l2": "inputs change every step"},
    }), flush=True)


def _hough(args):
    """64 binary 2048x2048 edge images (16 segments of 200-1500 px, +-1 px jitter,
    5% salt): Hough votes into 1024 x 2896 int32 bins, top-32 peaks per image,
    4 px bands, exact LMS of all 2048 sets.  Wall time per step of the whole
    (synchronous) call, images already in HBM."""
    import numpy as np
    import torch

    from paper_1510_01041_gb300 import build, datagen, lms
    build.build()
    imgs = torch.from_numpy(datagen.edge_images(64, 1)).cuda()
    for _ in range(args.warmup):
        lines = lms.hough_refine(imgs)
    torch.cuda.synchronize()
    lms.profile_read()
    lms.profile_enable(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lines = lms.hough_refine(imgs)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    lms.profile_enable(False)
    st = lms.profile_read()
    fitted = [ln for ln in lines if ln["fit"]["status"] == lms.LMS_OK]
    npts = [ln["npoints"] for ln in lines]
    print(json.dumps({
        "metric": "Hough + exact LMS line detection, images/sec", "value": 64 / dt, "unit": "images/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+int64",
        "data": "synthetic", "lines_per_sec": len(fitted) / dt,
        "config": {"workload": "64 x 2048x2048 edge images, 16 segments, 5% salt; 1024 theta x 2896 rho; "
                               "top-32, NMS +-5, 4 px band", "sets": len(lines),
                   "mean_points_per_set": float(np.mean(npts))},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in sorted(st.items(), key=lambda kv: -kv[1][0])},
    }), flush=True)


# The paper's Table 1 (one exact solve on random point sets; its GPU is
# named "GTX 720", a Kepler-class part), ms per solve: context only.
PAPER_TABLE1_MS = {128: 0.98, 256: 4.22, 512: 35.3}


def _table1(args):
    """The sizes of the paper's Table 1 (n = 128, 256, 512): one exact solve
    with the paper's own kernel layout (8x8-thread vertex blocks, one thread
    block and a shared-memory bitonic sort per vertex, reduction), with the
    per-slope warp kernel and with the kinetic sweep.  Device time per solve
    (CUDA events on the launching stream), inputs resident in HBM, L2 flushed
    (256 MB write) before every timed solve outside the events."""
    import numpy as np
    import torch

    from paper_1510_01041_gb300 import build, datagen, lms
    build.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = {}
    for n in sorted(PAPER_TABLE1_MS):
        x, y = datagen.line_with_outliers(n, 7)
        xt = torch.from_numpy(x).to(dev)
        yt = torch.from_numpy(y).to(dev)
        rows[n] = {"paper_table1_ms": PAPER_TABLE1_MS[n]}
        ref = None
        for algo in ("paper", "plain", "sweep"):
            out = torch.empty(lms.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            for _ in range(args.warmup):
                lms.fit(xt, yt, 0, algo, out=out)
            torch.cuda.synchronize()
            tot = 0.0
            for _ in range(args.steps):
                flush.fill_(1)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lms.fit(xt, yt, 0, algo, out=out)
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            r = lms.decode(out)[0]
            got = tuple(r[k] for k in ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "i", "j"))
            ref = ref or got
            if got != ref:
                raise SystemExit(f"n={n}: {algo} disagrees: {got} vs {ref}")
            rows[n][algo + "_ms"] = tot / args.steps
    v = 1000.0 / rows[512]["paper_ms"]
    print(json.dumps({
        "metric": "exact LMS solves/sec at n=512 with the paper's kernel layout (Table 1 sizes)",
        "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": rows[512]["paper_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": v / (1000.0 / PAPER_TABLE1_MS[512]), "dtype": "int64", "data": "synthetic",
        "config": {"workload": "one exact fit of line_with_outliers at n = 128, 256, 512 (paper Table 1 sizes)",
                   "l2": "flushed before every timed solve (256 MB write, outside the events)",
                   "baseline": "paper Table 1, GTX-class GPU of 2015 (context)"},
        "rows_ms": {str(k): v2 for k, v2 in rows.items()},
    }), flush=True)


def _line_errors(lines, truth, n_theta, n_rho, cs):
    """Slope errors (percent of |true slope|) of the Hough peak line (SHT),
    least squares (OLS) and exact LMS on the peak's band points, each in the
    fit's frame (x and y swapped for near-vertical peaks), one line per image."""
    import numpy as np
    out = {"sht": [], "ols": [], "lms": []}
    for b, ln in enumerate(lines):
        if ln["theta_index"] < 0 or ln["fit"]["status"] != 0:
            continue
        s_true, c_true = truth[b]
        t = ln["theta_index"]
        c, sn = float(cs[t, 0]), float(cs[t, 1])
        rho_c = ln["rho_index"] - n_rho // 2 + 0.5
        if ln["transposed"]:
            s_ref = 1.0 / s_true                   # x = y / s - c / s
            s_sht = -sn / c
        else:
            s_ref = s_true
            s_sht = -c / sn
        for k, v in (("sht", s_sht), ("ols", ln["ols_theta1"]), ("lms", ln["fit"]["theta1"])):
            out[k].append(100.0 * abs(v - s_ref) / abs(s_ref))
    return {k: (float(np.median(v)) if v else None) for k, v in out.items()}


def _accuracy(args):
    """The paper's line-detection experiments (Sec. 5.1) on seeded synthetic
    1024x1024 images with one segment whose pixels are kept with probability
    0.5 plus salt noise: slope error of the Hough peak line (SHT), of least
    squares on the peak's supporting points (OLS) and of the exact LMS of the
    same points, (a) over accumulator resolutions (theta bin width with a
    matching support band) at noise 0.001, (b) over noise probabilities
    0.001 .. 0.006 at 1 degree / 4 px.  Median over 48 images per setting."""
    import numpy as np
    import torch

    from paper_1510_01041_gb300 import build, datagen, lms
    build.build()
    n_img, size = 48, 1024
    n_rho = 2 * int(math.ceil(math.hypot(size, size) / 2)) + 2

    def tables(n_theta):
        th = np.pi * np.arange(n_theta, dtype=np.float64) / n_theta
        return np.stack([np.cos(th), np.sin(th)], axis=1).astype(np.float32)

    def run(noise, dtheta_deg, band, seed):
        imgs, truth = datagen.single_line_images(n_img, seed, size=size, noise=noise)
        n_theta = int(round(180.0 / dtheta_deg))
        cs = tables(n_theta)
        lines = lms.hough_refine(torch.from_numpy(imgs).cuda(), n_theta, n_rho, 1, band, 5, 5,
                                 cos_sin=torch.from_numpy(cs).cuda())
        return _line_errors(lines, truth, n_theta, n_rho, cs)

    res_rows = {}
    for dth, band in ((0.25, 1.0), (0.5, 2.0), (1.0, 4.0), (2.0, 8.0), (4.0, 16.0)):
        res_rows[f"dtheta={dth}deg,band={band}px"] = run(0.001, dth, band, 11)
    noise_rows = {}
    for p in (0.001, 0.002, 0.003, 0.004, 0.005, 0.006):
        noise_rows[f"noise={p}"] = run(p, 1.0, 4.0, 12)
    v = noise_rows["noise=0.001"]["lms"]
    print(json.dumps({
        "metric": "median line slope error (percent), exact LMS on Hough peak support, synthetic 1024^2 images",
        "value": v, "unit": "percent", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "48 images 1024x1024 per setting: one segment (pixels kept with p=0.5) + salt noise",
                   "paper_context": "Sec. 5.1: LMS 0.37% vs OLS 12.4% over resolutions; LMS < 0.14% below "
                                    "noise 0.004, 3.38% at 0.004 (other images, other detector)"},
        "over_resolution": res_rows, "over_noise": noise_rows,
    }), flush=True)


def _subsample(args):
    """Random subsampling of each peak's supporting points before the exact
    LMS (Sec. 5: a further speed-up the paper suggests): the 64-image Hough
    workload with at most M points per set, M = all, 512, 256, 128, 64; time
    per step and the median / 95th percentile angle between each subsampled
    fit and the full fit."""
    import numpy as np
    import torch

    from paper_1510_01041_gb300 import build, datagen, lms
    build.build()
    imgs = torch.from_numpy(datagen.edge_images(64, 1)).cuda()
    rows = {}
    full = None
    for M in (0, 512, 256, 128, 64):
        for _ in range(args.warmup):
            lines = lms.hough_refine(imgs, max_points=M, sample_seed=7)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            lines = lms.hough_refine(imgs, max_points=M, sample_seed=7)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        ang = np.array([math.atan(ln["fit"]["theta1"]) if ln["fit"]["status"] == 0 else np.nan for ln in lines])
        if full is None:
            full = ang
        d = np.degrees(np.abs(ang - full))
        d = d[np.isfinite(d)]
        rows[str(M or "all")] = {"ms_per_step": dt * 1e3, "median_points_fitted": float(np.median([ln["nfit"] for ln in lines])),
                                 "angle_dev_deg_median": float(np.median(d)), "angle_dev_deg_p95": float(np.percentile(d, 95))}
    print(json.dumps({
        "metric": "Hough + LMS images/sec with supporting points subsampled to at most 128 per line",
        "value": 64 / (rows["128"]["ms_per_step"] / 1e3), "unit": "images/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rows["128"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+int64", "data": "synthetic",
        "config": {"workload": "64 x 2048x2048 edge images, 16 segments, 5% salt; 1024 x 2896 bins; top-32, 4 px band",
                   "sampling": "Bernoulli per point, rate M / band size, SplitMix64 on (seed, set, rank)"},
        "rows": rows,
    }), flush=True)


def _timed(fit, steps, warmup, flush, stream, barrier):
    """Per-step CUDA-event device time of `fit(k)` for steps warmup..warmup+steps-1."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    for k in range(steps):
        s = warmup + k
        flush.fill_(s & 0xff)
        ev[k][0].record(stream)
        fit(s)
        ev[k][1].record(stream)
    barrier()
    return sum(a.elapsed_time(b) for a, b in ev)


def batched_short(steps: int, warmup: int):
    """The batch workload (4096 uneven sets) with a fixed plan (plain kernel up
    to 128 points, 48 streams, branch-and-bound from 512 points), captured
    into one CUDA graph; each step replays it on a fresh batch already in HBM
    (y coordinates of another seed), timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1510_01041_gb300 import datagen, lms
    dev = torch.device("cuda", torch.cuda.current_device())
    x0, y0, off = datagen.batch(4096, 5000)
    # a second batch of the same set sizes: every y moved by a seeded U{-2..2}
    y1 = (y0.astype(np.int64) + datagen.Stream(5001).integers(-2, 3, y0.size)).clip(-32768, 32767).astype(np.int16)
    xt, yt, ot = (torch.from_numpy(a).to(dev) for a in (x0, y0, off))
    ys = [torch.from_numpy(y0).to(dev), torch.from_numpy(y1).to(dev)]
    plan = lms.BatchPlan(off, plain_max_n=128, streams=48, bnb_min_n=512)
    out = torch.empty((4096, lms.RESULT_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    plan.fit(xt, yt, ot, out=out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(xt, yt, ot, out=out, stream=s)
    for k in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    ms = 0.0
    for k in range(steps):
        yt.copy_(ys[k % len(ys)])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    res = lms.decode(out)
    assert all(r["status"] in (lms.LMS_OK, lms.LMS_ERR_VERTICAL) for r in res)
    sizes = np.diff(off)
    slopes = int(np.sum(sizes * (sizes - 1) // 2))
    v = 4096 * steps / (ms / 1000.0)
    return {"value": v, "unit": UNIT, "ms_per_step": ms / steps, "candidate_slopes_per_sec": v / 4096 * slopes,
            "steps": steps, "warmup": warmup,
            "workload": "4096 sets, n log-uniform [64,4096], outliers U(0,0.45), angle U(-1.5,1.5)",
            "plan": "plain kernel <= 128 points, 48 streams, branch-and-bound >= 512 points, one CUDA graph"}


def hough_short(steps: int, warmup: int):
    """The line-detection workload: 64 binary 2048x2048 edge images, Hough
    votes into 1024 x 2896 bins, top-32 peaks, 4 px bands, exact LMS of all
    2048 sets; wall time of the whole (synchronous) call, images in HBM."""
    import torch

    from paper_1510_01041_gb300 import datagen, lms
    imgs = torch.from_numpy(datagen.edge_images(64, 1)).cuda()
    for _ in range(warmup):
        lms.hough_refine(imgs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        lines = lms.hough_refine(imgs)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    fitted = sum(1 for ln in lines if ln["fit"]["status"] == lms.LMS_OK)
    return {"value": 64 / dt, "unit": "images/s", "ms_per_step": dt * 1e3, "lines_per_sec": fitted / dt,
            "steps": steps, "warmup": warmup,
            "workload": "64 x 2048x2048 edge images, 16 segments, 5% salt; 1024 theta x 2896 rho; top-32, 4 px band"}


def node_bound_ops(n: int) -> int:
    """Algorithmic int32 instruction-equivalents of one slope interval's lower
    bound: projections of all points at both interval ends (4n, 4 ops each:
    a 32x32->64 multiply-add, shift, subtract, min/max), two comparison sorts
    of n 32-bit keys (n ceil(log2 n) merge steps each, 4 ops a step: compare,
    select the value, advance an index, select the new head) and one scan of
    the n - h + 1 windows (3 ops each)."""
    lg = max(1, math.ceil(math.log2(n)))
    return 4 * n * 4 + 2 * n * lg * 4 + 3 * n


# Algorithmic work per unit, int32 instruction-equivalents:
#   sweep        per event swept (SWEEP_INT_OPS_PER_EVENT)
#   node_bounds  per slope interval bounded (node_bound_ops)
# (The restricted pair pass is a band scan whose work follows the pairs its
# bands meet, which no statistic reports; it has no modeled entry.)


def _roof(stage, stages, units_per_fit, ops_per_unit, fits, peak_tops, mhz_basis, traffic=None):
    ms, launches = stages.get(stage, (0.0, 0))
    if not launches or units_per_fit <= 0:
        return None
    per_launch_s = ms / launches / 1000.0
    units = units_per_fit * fits / launches
    achieved = units * ops_per_unit / per_launch_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s (int32)",
            "frac": achieved / peak_tops, "traffic": traffic, "traffic_unit": "bytes per launch (ncu)",
            "stage": stage, "kernel_ms": per_launch_s * 1e3, "launches_per_fit": launches / fits,
            "units_per_launch": units, "ops_per_unit": ops_per_unit, "peak_basis": mhz_basis}


# Kernels of the timed paths: the stage name the library's profiler uses,
# the kernel, and its DRAM traffic per launch (dram__bytes_read.sum +
# dram__bytes_write.sum) from the ncu captures summarised under profiles/;
# a kernel changed after its capture has no entry.
KERNEL_OF_STAGE = {"sweep": "k_sweep", "node_bounds": "k_node_lb"}
DRAM_BYTES = {"k_node_lb": 152_320, "k_sweep": 386_048, "k_sweep_plain": 194_637_824}


def _instances(seeds):
    from paper_1510_01041_gb300 import datagen
    return [datagen.sloped(N_POINTS, s, OUTLIER_FRAC, phi_max=PHI_MAX)[:2] for s in seeds]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the short batch and Hough lines")
    ap.add_argument("--breakdown", action="store_true", help="per-stage times to stderr")
    ap.add_argument("--workload", choices=["single", "batched", "hough", "table1", "accuracy", "subsample"],
                    default="single",
                    help="single: n=8192 fit (default); batched: 4096 uneven sets in one graph; "
                         "hough: 64 edge images, Hough peaks refined by exact LMS; table1: the paper's "
                         "kernel layout, the warp kernel and the sweep at n = 128, 256, 512; accuracy: SHT / OLS / LMS "
                         "slope errors on synthetic single-line images; subsample: Hough + LMS with the supporting "
                         "points randomly subsampled")
    args = ap.parse_args()
    if args.impl == "reference":
        _reference_arm(args)
        return
    if args.workload == "batched":
        _batched(args)
        return
    if args.workload == "hough":
        _hough(args)
        return
    if args.workload == "table1":
        _table1(args)
        return
    if args.workload == "accuracy":
        _accuracy(args)
        return
    if args.workload == "subsample":
        _subsample(args)
        return

    import numpy as np
    import torch

    from paper_1510_01041_gb300 import build, datagen, lms

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    total = args.warmup + args.steps
    seeds = rank_seeds(rank, total)
    host = _instances(seeds)
    # the previous workload (fixed slope 0.7, 40% outliers) beside it
    host2 = [datagen.line_with_outliers(N_POINTS, s, 0.4) for s in seeds]
    xs = [torch.from_numpy(h[0]).to(dev) for h in host]
    ys = [torch.from_numpy(h[1]).to(dev) for h in host]
    xs2 = [torch.from_numpy(h[0]).to(dev) for h in host2]
    ys2 = [torch.from_numpy(h[1]).to(dev) for h in host2]
    R = lms.RESULT_DTYPE.itemsize
    outs = {k: torch.empty((total, R), dtype=torch.uint8, device=dev)
            for k in ("learned", "quantile", "plain", "learned2", "plain2")}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lms.reserve(N_POINTS, algorithm="bnb")
    net = lms.pretrained()
    # measured int32 peaks of this GPU (outside every timed region)
    peak_addxor = lms.measure_int_peak(0, 20000) / 1e12
    peak_imad = lms.measure_int_peak(1, 20000) / 1e12

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # the timed arms ask for no statistics (a fit with statistics waits for
    # its result); a separate untimed pass below reads them
    stats = {"learned": [], "quantile": []}
    arms = {
        "learned": lambda s: net.fit(xs[s], ys[s], 0, out=outs["learned"][s], stats=False),
        "quantile": lambda s: lms.fit_bnb(xs[s], ys[s], 0, None, out=outs["quantile"][s], seed_mode="quantiles",
                                          stats=False),
        "plain": lambda s: lms.fit(xs[s], ys[s], 0, "sweep", out=outs["plain"][s]),
        "learned2": lambda s: net.fit(xs2[s], ys2[s], 0, out=outs["learned2"][s]),
        "plain2": lambda s: lms.fit(xs2[s], ys2[s], 0, "sweep", out=outs["plain2"][s]),
    }
    for s in range(args.warmup):
        flush.fill_(s & 0xff)
        for f in arms.values():
            f(s)
    barrier()
    # The two branch-and-bound arms of the headline workload are timed as
    # CUDA-graph replays: each timed step's fit (its own input and output
    # buffers, no statistics) is captured once here, so the timed region
    # runs the same kernels without the host's launch calls between them.
    # The library counts its launches on the host, so each graph's launches
    # are counted while it is captured.
    graphed, graph_launches = {}, {}
    cap = torch.cuda.Stream(dev)
    for k in ("learned", "quantile"):
        gs, nl = [], []
        for s in range(args.warmup, total):
            g = torch.cuda.CUDAGraph()
            cap.wait_stream(stream)
            l0 = lms.launch_count()
            with torch.cuda.stream(cap):
                with torch.cuda.graph(g, stream=cap):
                    arms[k](s)
            nl.append(lms.launch_count() - l0)
            gs.append(g)
        stream.wait_stream(cap)
        graphed[k] = (lambda gs: lambda s: gs[s - args.warmup].replay())(gs)
        graph_launches[k] = sum(nl)
    barrier()
    ms, stages = {}, {}
    # timed passes without the library's per-launch profiling events
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        ms["learned"] = _timed(graphed["learned"], args.steps, args.warmup, flush, stream, barrier)
        launches = graph_launches["learned"]
        wall = time.perf_counter() - wall0
        ms["quantile"] = _timed(graphed["quantile"], args.steps, args.warmup, flush, stream, barrier)
        for k in ("plain", "learned2", "plain2"):
            ms[k] = _timed(arms[k], args.steps, args.warmup, flush, stream, barrier)
    # a second pass over the same steps with CUDA events around every launch,
    # on the stream it runs on: per-kernel times for the stage table and the
    # roofline (the events add a little time between launches, not inside them)
    lms.profile_read()
    lms.profile_enable(True)
    for k in ("learned", "quantile", "plain"):
        _timed(arms[k], args.steps, args.warmup, flush, stream, barrier)
        stages[k] = lms.profile_read()
    lms.profile_enable(False)
    # statistics of the branch-and-bound fits (untimed)
    for s in range(args.warmup, args.warmup + args.steps):
        stats["learned"].append(net.fit(xs[s], ys[s], 0, out=outs["learned"][s])[1])
        stats["quantile"].append(lms.fit_bnb(xs[s], ys[s], 0, None, out=outs["quantile"][s],
                                             seed_mode="quantiles")[1])
    ms = {k: max_over_ranks(v, dev) for k, v in ms.items()}
    res = {k: lms.decode(v)[args.warmup:] for k, v in outs.items()}
    keys = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j", "theta1", "theta2", "med_sq")
    for a, b, c in zip(res["learned"], res["quantile"], res["plain"]):
        if a["status"] != lms.LMS_OK or not (tuple(a[k] for k in keys) == tuple(b[k] for k in keys)
                                             == tuple(c[k] for k in keys)):
            raise SystemExit(f"learned, quantile-seeded and plain fits disagree: {a} {b} {c}")
    for a, c in zip(res["learned2"], res["plain2"]):
        if a["status"] != lms.LMS_OK or tuple(a[k] for k in keys) != tuple(c[k] for k in keys):
            raise SystemExit(f"learned and plain fits disagree (line_with_outliers): {a} {c}")

    # end to end through the public C ABI with host buffers: lms_fit_learned_host
    # copies the points in, fits and copies the 88-byte result out every step
    pin_x = [torch.from_numpy(h[0]).pin_memory() for h in host]
    pin_y = [torch.from_numpy(h[1]).pin_memory() for h in host]
    hres = torch.zeros(R, dtype=torch.uint8).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        s = args.warmup + k
        net.fit_host(pin_x[s], pin_y[s], 0, out=hres, stats=False)
        r = lms.decode(hres)[0]
        if tuple(r[q] for q in keys) != tuple(res["learned"][k][q] for q in keys):
            raise SystemExit("host-buffer learned fit disagrees with the device-buffer fit")
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)

    slopes = N_POINTS * (N_POINTS - 1) // 2
    rate = {k: job_rate(args.steps, ws, v) for k, v in ms.items()}
    csum = clk.summary()
    mhz = csum.get("sm_mhz") or 0.0
    basis = (f"measured: lms_measure_int_peak kind 0 (int32 add/xor chains, full occupancy), "
             f"{peak_addxor:.2f} Tops/s; kind 1 (multiply-add) {peak_imad:.2f} Tops/s")
    peak = max(peak_addxor, peak_imad)
    mean = lambda arm, k: float(np.mean([st[k] for st in stats[arm]])) if stats[arm] else 0.0
    roofs = {}
    for arm, st in (("learned", stages["learned"]),):
        roofs["sweep"] = _roof("sweep", st, mean(arm, "events_swept"), SWEEP_INT_OPS_PER_EVENT, args.steps, peak,
                               basis, DRAM_BYTES.get("k_sweep"))
        roofs["node_bounds"] = _roof("node_bounds", st, mean(arm, "nodes_evaluated"), node_bound_ops(N_POINTS),
                                     args.steps, peak, basis, DRAM_BYTES.get("k_node_lb"))
    # the plain path's sweep kernel: every pair with distinct x is an event
    events = [int(np.sum(np.triu(np.not_equal.outer(h[0], h[0]), 1))) for h in host[args.warmup:]]
    plain_sweep_roof = _roof("sweep", stages["plain"], float(np.mean(events)), SWEEP_INT_OPS_PER_EVENT, args.steps,
                             peak, basis, DRAM_BYTES.get("k_sweep_plain"))
    modeled = {k: v for k, v in roofs.items() if v}
    dom = max(modeled, key=lambda k: stages["learned"][k][0]) if modeled else None
    roof = None
    if dom:
        roof = dict(modeled[dom])
        roof["kernel"] = KERNEL_OF_STAGE[dom] + " (learned-seeded path, dominant modeled kernel)"
    if plain_sweep_roof:
        plain_sweep_roof["kernel"] = "k_sweep (plain path, every event)"

    def arm_line(k, extra=None):
        d = {"value": rate[k], "unit": UNIT, "ms_per_step": ms[k] / args.steps,
             "candidate_slopes_per_sec": rate[k] * slopes}
        d.update(extra or {})
        return d

    line = {
        "metric": METRIC, "value": rate["learned"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms["learned"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "candidate_slopes_per_sec": rate["learned"] * slopes,
        "learned": arm_line("learned", {"events_swept_mean": mean("learned", "events_swept"),
                                        "nodes_evaluated_mean": mean("learned", "nodes_evaluated"),
                                        "levels_mean": mean("learned", "levels"),
                                        "buckets_swept_mean": mean("learned", "buckets_swept"),
                                        "upper_bound_mean": mean("learned", "upper_bound"),
                                        "algorithm": "set-network seed + branch-and-bound"}),
        "quantile_bnb": arm_line("quantile", {"events_swept_mean": mean("quantile", "events_swept"),
                                              "nodes_evaluated_mean": mean("quantile", "nodes_evaluated"),
                                              "levels_mean": mean("quantile", "levels"),
                                              "buckets_swept_mean": mean("quantile", "buckets_swept"),
                                              "upper_bound_mean": mean("quantile", "upper_bound"),
                                              "algorithm": "branch-and-bound seeded at sample quantiles "
                                                           "(the method without the network)"}),
        "plain": arm_line("plain", {"algorithm": "kinetic sweep, every slope"}),
        "events_total_mean": mean("learned", "events_total"),
        "line_40pct": {"workload": "line_with_outliers: slope 0.7, 40% outliers, n=8192",
                       "learned": arm_line("learned2"), "plain": arm_line("plain2")},
        "config": {"workload": WORKLOAD, "n": N_POINTS, "h": N_POINTS // 2 + 1,
                   "algorithm": "learned-seeded branch-and-bound + sweep of surviving slopes",
                   "l2": "flushed before every step (256 MB write, outside the timed events)",
                   "launch": "learned and quantile-seeded fits: one CUDA graph per step, captured after "
                             "the warm-up and replayed; plain sweep and the 40% line workload: direct calls",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": args.steps * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * 2 * N_POINTS,
                "d2h_bytes_per_step": R,
                "api": "lms_fit_learned_host (C ABI, pinned host buffers, copies in the timed region)",
                "l2": "not flushed: back-to-back calls, wall clock around copies, fit and result read"},
        "gpu_launches": launches,
        "clocks": {k: csum.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "roofline": roof,
        "roofline_kernels": {"learned_path": modeled, "plain_path_sweep": plain_sweep_roof},
        "int_peak_tops": {"add_xor": peak_addxor, "imad": peak_imad, "sm_mhz_during_run": mhz,
                          "sms": props.multi_processor_count},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in
                              sorted(stages["learned"].items(), key=lambda kv: -kv[1][0])},
        "plain_stage_ms_per_step": {k: v[0] / args.steps for k, v in
                                    sorted(stages["plain"].items(), key=lambda kv: -kv[1][0])},
        "wall_s": wall,
    }
    if rank == 0 and ws == 1 and not args.no_extra:
        line["batched"] = batched_short(3, 2)
        line["hough"] = hough_short(3, 1)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, o = _cpu_baseline(*host[args.warmup])
        r = res["learned"][0]
        cb["agrees_with_gpu"] = (r["w_num"], r["w_den"], r["s_num"], r["s_den"], r["t_num"], r["i"], r["j"]) == (
            o.w_num, o.w_den, o.s_num, o.s_den, o.t_num, o.i, o.j)
        line["cpu_baseline"] = cb
    if args.breakdown and rank == 0:
        for name in ("learned", "quantile", "plain"):
            for k, v in sorted(stages[name].items(), key=lambda kv: -kv[1][0]):
                print(f"  {name:8s} {k:14s} {v[0] / args.steps:9.3f} ms/step  launches {v[1]}", file=sys.stderr)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
