"""CPU oracle of the learned slope proposal's set network (float64 numpy).

TEST INFRASTRUCTURE ONLY.  Independent of the CUDA kernels: plain numpy
forward and backward of

    per point p:  h1 = relu(W1 [xn, yn] + b1)      (64)
                  h2 = relu(W2 h1 + b2)            (64)
    g = max over points of h2 (per channel; ties -> smallest point index)
    h3 = relu(W3 g + b3)                            (32)
    (phi, b) = W4 h3 + b4

with every parameter first rounded to bfloat16 (round to nearest even), as
the device computes with BF16 weights.  Frame of a set: centre of the
bounding box, scale = half the larger side (at least 1).
Loss = mean over sets of (phi - phi*)^2 + lam (b - b*)^2.
"""
from __future__ import annotations

import numpy as np

H1, H2, H3, NOUT = 64, 64, 32, 2
SHAPES = [("W1", (H1, 2)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)),
          ("W3", (H3, H2)), ("b3", (H3,)), ("W4", (NOUT, H3)), ("b4", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), back as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def frame(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    cx = 0.5 * (x.min() + x.max())
    cy = 0.5 * (y.min() + y.max())
    sc = max(1.0, 0.5 * max(x.max() - x.min(), y.max() - y.min()))
    return cx, cy, sc


def forward(flat, x, y):
    """Returns (phi, b, cache) for one set."""
    P = unpack(bf16_round(np.asarray(flat, np.float32)).astype(np.float64))
    cx, cy, sc = frame(x, y)
    X = np.stack([(np.asarray(x, np.float64) - cx) / sc, (np.asarray(y, np.float64) - cy) / sc], axis=1)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    arg = np.argmax(h2, axis=0)            # first maximum = smallest index
    g = h2[arg, np.arange(H2)]
    z3 = P["W3"] @ g + P["b3"]
    h3 = np.maximum(z3, 0.0)
    out = P["W4"] @ h3 + P["b4"]
    cache = dict(P=P, X=X, z1=z1, h1=h1, z2=z2, arg=arg, g=g, z3=z3, h3=h3)
    return out[0], out[1], cache


def loss_and_grad(flat, sets, targets, lam):
    """Mean loss over sets and its gradient w.r.t. the (bf16-rounded) parameters."""
    B = len(sets)
    grads = {name: np.zeros(shp) for name, shp in SHAPES}
    L = 0.0
    for (x, y), (tphi, tb) in zip(sets, targets):
        phi, b, c = forward(flat, x, y)
        e0, e1 = phi - tphi, b - tb
        L += (e0 * e0 + lam * e1 * e1) / B
        dout = np.array([2 * e0 / B, 2 * lam * e1 / B])
        P = c["P"]
        grads["W4"] += np.outer(dout, c["h3"])
        grads["b4"] += dout
        dz3 = (P["W4"].T @ dout) * (c["z3"] > 0)
        grads["W3"] += np.outer(dz3, c["g"])
        grads["b3"] += dz3
        dg = P["W3"].T @ dz3
        for ch in range(H2):
            p = c["arg"][ch]
            dz2 = dg[ch] if c["g"][ch] > 0 else 0.0
            grads["b2"][ch] += dz2
            if dz2 == 0.0:
                continue
            grads["W2"][ch] += dz2 * c["h1"][p]
            dz1 = P["W2"][ch] * dz2 * (c["z1"][p] > 0)
            grads["W1"] += np.outer(dz1, c["X"][p])
            grads["b1"] += dz1
    flatg = np.concatenate([grads[name].ravel() for name, _ in SHAPES])
    return L, flatg


def loss_only(flat, sets, targets, lam):
    """Loss with parameters used as given (no bf16 rounding): for finite differences."""
    P = unpack(flat)
    B = len(sets)
    L = 0.0
    for (x, y), (tphi, tb) in zip(sets, targets):
        cx, cy, sc = frame(x, y)
        X = np.stack([(np.asarray(x, np.float64) - cx) / sc, (np.asarray(y, np.float64) - cy) / sc], axis=1)
        h1 = np.maximum(X @ P["W1"].T + P["b1"], 0.0)
        h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
        g = h2.max(axis=0)
        h3 = np.maximum(P["W3"] @ g + P["b3"], 0.0)
        o = P["W4"] @ h3 + P["b4"]
        L += ((o[0] - tphi) ** 2 + lam * (o[1] - tb) ** 2) / B
    return L


def targets_from_fit(x, y, theta1, theta2):
    """(angle, normalised intercept) of an LMS line in the set's frame."""
    cx, cy, sc = frame(x, y)
    return float(np.arctan(theta1)), float((theta2 - cy + theta1 * cx) / sc)
