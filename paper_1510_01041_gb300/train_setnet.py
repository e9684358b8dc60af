"""Train the learned slope proposal on instances the method itself solves.

Every training set comes from the seeded generator (random slope angle in
(-1.4, 1.4), integer intercept, noise +-3, outlier fraction U(0, 0.45),
n log-uniform in [256, 8192]); its target is the exact LMS line found by this
library (lms_fit), expressed as (angle, normalised intercept) in the set's
bounding-box frame.  Training runs the library's own forward, backward and
Adam kernels (lms_setnet_train_step).  The result is written to
weights/setnet.bin together with a JSON summary.

    python -m paper_1510_01041_gb300.train_setnet [--sets 4096] [--steps 3000]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import build, datagen, lms

HERE = os.path.dirname(os.path.abspath(__file__))


def frame(x, y):
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    cx = 0.5 * (x.min() + x.max())
    cy = 0.5 * (y.min() + y.max())
    sc = max(1.0, 0.5 * max(x.max() - x.min(), y.max() - y.min()))
    return cx, cy, sc


def make_sets(count: int, seed: int, n_min: int, n_max: int):
    st = datagen.Stream(seed)
    u = st.uniform(count)
    fr = st.uniform(count) * 0.45
    sizes = np.floor(n_min * (n_max / n_min) ** u).astype(np.int64)
    sets = []
    for k in range(count):
        x, y, _ = datagen.sloped(int(sizes[k]), seed * 7777 + k, float(fr[k]), phi_max=1.4)
        sets.append((x, y))
    return sets


def solve(sets, device):
    """Exact LMS of every set with this library (branch-and-bound above 1024 points)."""
    import torch
    out = []
    for x, y in sets:
        xt, yt = torch.from_numpy(x).to(device), torch.from_numpy(y).to(device)
        res = lms.fit_bnb(xt, yt)[0] if x.size > 1024 else lms.fit(xt, yt)
        r = lms.decode(res)[0]
        cx, cy, sc = frame(x, y)
        out.append((math.atan(r["theta1"]), (r["theta2"] - cy + r["theta1"] * cx) / sc))
    return np.array(out, dtype=np.float32)


def csr(sets, idx, device):
    import torch
    xs = np.concatenate([sets[k][0] for k in idx])
    ys = np.concatenate([sets[k][1] for k in idx])
    off = np.zeros(len(idx) + 1, dtype=np.int64)
    off[1:] = np.cumsum([sets[k][0].size for k in idx])
    return (torch.from_numpy(xs).to(device), torch.from_numpy(ys).to(device), torch.from_numpy(off).to(device))


def angle_errors(net, sets, targets, device, batch=64):
    """Absolute angle errors (radians) of the network's predictions."""
    errs = []
    for s in range(0, len(sets), batch):
        idx = list(range(s, min(len(sets), s + batch)))
        x, y, off = csr(sets, idx, device)
        pred = net.forward(x, y, off).cpu().numpy()
        errs.append(np.abs(pred[:, 0] - targets[idx, 0]))
    return np.concatenate(errs)


def angle_error(net, sets, targets, device, batch=64):
    return float(np.mean(angle_errors(net, sets, targets, device, batch)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=4096)
    ap.add_argument("--val", type=int, default=256)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lam", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--n-max", type=int, default=8192)
    ap.add_argument("--out", default=lms.WEIGHTS)
    args = ap.parse_args()
    import torch
    build.build()
    device = torch.device("cuda", 0)
    t0 = time.time()
    train = make_sets(args.sets, 1000 + args.seed, 256, args.n_max)
    val = make_sets(args.val, 9000 + args.seed, 256, args.n_max)
    ttrain = solve(train, device)
    tval = solve(val, device)
    t_solve = time.time() - t0
    net = lms.SetNet(args.seed)
    base_err = angle_error(net, val, tval, device)
    rng = np.random.default_rng(args.seed)
    tt = torch.from_numpy(ttrain).to(device)
    loss = torch.zeros(1, device=device)
    t1 = time.time()
    hist = []
    for step in range(args.steps):
        idx = rng.choice(len(train), args.batch, replace=False)
        x, y, off = csr(train, idx, device)
        targets = tt[torch.from_numpy(idx).to(device)].contiguous()
        lr = args.lr * (0.5 * (1 + math.cos(math.pi * step / args.steps)))
        net.train_step(x, y, off, targets, args.lam, lr, loss=loss)
        if step % 250 == 0 or step == args.steps - 1:
            hist.append((step, float(loss.item())))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    errs = angle_errors(net, val, tval, device)
    err = float(np.mean(errs))
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    net.save(args.out)
    summary = dict(train_sets=args.sets, val_sets=args.val, n_range=[256, args.n_max], steps=args.steps,
                   batch=args.batch, lr=args.lr, lam=args.lam, seed=args.seed,
                   val_angle_mae_rad_untrained=base_err, val_angle_mae_rad=err,
                   val_angle_err_rad_median=float(np.median(errs)),
                   val_angle_err_rad_p90=float(np.percentile(errs, 90)),
                   loss_history=hist, solve_seconds=t_solve, train_seconds=t_train)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
