"""Autotuner for batched fits: picks the size threshold between the plain
kernel classes and the sweep, the number of sweep streams and the size from
which sets take the branch-and-bound instead of the sweep, by timing
CUDA-graph replays of a batch plan on the caller's own sets.  Results are
cached per (device name, size mix) in autotune_cache.json next to this
file, or in the file $LMS_AUTOTUNE_CACHE names.

    from paper_1510_01041_gb300 import autotune
    plan, cfg = autotune.tuned_plan(offsets, x, y, offsets_dev)
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import lms

# The cache file: $LMS_AUTOTUNE_CACHE if set, else next to this module; a
# cache that cannot be written is reported by a warning and tuning still works.
CACHE = os.environ.get("LMS_AUTOTUNE_CACHE") or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                             "autotune_cache.json")
PLAIN_MAX = (64, 128, 256)
STREAMS = (8, 16, 32, 48)
BNB_MIN = (384, 512, 768, 1536, -1)   # -1: every large set takes the sweep of every slope


def _key(offsets, device_name):
    """Device, set count, total points, total candidate pairs and a histogram
    of set sizes at eighth-octave resolution: batches that differ in how
    their work is spread over sizes get different keys; the order of the
    sets does not matter."""
    sizes = np.diff(np.asarray(offsets, dtype=np.int64))
    hist = np.histogram(np.log2(np.maximum(sizes, 2)), bins=128, range=(1, 17))[0]
    pairs = int(np.sum(sizes * (sizes - 1) // 2))
    h = hashlib.sha1(hist.tobytes() + device_name.encode()).hexdigest()[:16]
    return f"v2:{device_name}:{sizes.size}:{int(sizes.sum())}:{pairs}:{h}"


def _time_plan(plan, x, y, od, reps=2):
    import torch
    out = torch.empty((plan.B, lms.RESULT_DTYPE.itemsize), dtype=torch.uint8, device=x.device)
    plan.fit(x, y, od, out=out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(x, y, od, out=out, stream=s)
    g.replay()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        g.replay()
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / reps, g, out


def tune(offsets, x, y, offsets_dev, candidates=None):
    """Time candidate plans (plain_max_n, streams, bnb_min_n); returns the
    best config.  Coordinate search: the plain threshold and stream count at
    the default branch-and-bound size, then the branch-and-bound size at the
    best of those (or every given candidate)."""
    import torch
    results = []

    def run(pm, ns, bm):
        plan = lms.BatchPlan(offsets, plain_max_n=pm, streams=ns, bnb_min_n=bm)
        dt, _, _ = _time_plan(plan, x, y, offsets_dev, reps=1)
        results.append(dict(plain_max_n=pm, streams=ns, bnb_min_n=bm, seconds=dt))
        del plan
        torch.cuda.synchronize()

    if candidates:
        for c in candidates:
            run(*c)
    else:
        for pm in PLAIN_MAX:
            for ns in STREAMS:
                run(pm, ns, 0)
        b = min(results, key=lambda r: r["seconds"])
        for bm in BNB_MIN:
            run(b["plain_max_n"], b["streams"], bm)
    best = min(results, key=lambda r: r["seconds"])
    return best, results


def tuned_plan(offsets, x, y, offsets_dev, use_cache=True):
    import torch
    key = _key(offsets, torch.cuda.get_device_name(x.device))
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        cfg = cache[key]
    else:
        cfg, _ = tune(offsets, x, y, offsets_dev)
        cache[key] = cfg
        try:
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError as e:
            import warnings
            warnings.warn(f"autotune cache {CACHE} not written ({e}); set LMS_AUTOTUNE_CACHE to a writable path")
    return lms.BatchPlan(offsets, plain_max_n=cfg["plain_max_n"], streams=cfg["streams"],
                         bnb_min_n=cfg.get("bnb_min_n", 0)), cfg
