"""The set-network oracle's backward pass equals finite differences of its
loss (float64), and bf16 rounding matches the IEEE round-to-nearest-even rule."""
import numpy as np

from oracle import setnet


def test_bf16_rounding_rule():
    v = np.array([1.0, 1.00390625, 1.0078125, 1.01171875, -3.140625, 65504.0], dtype=np.float32)
    r = setnet.bf16_round(v)
    # 1 + 2^-8 is half-way between 1 and 1 + 2^-7: ties to even -> 1
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == np.float32(1.0078125)
    # 1 + 3 * 2^-8 is half-way between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert r[3] == np.float32(1.015625)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2.0 ** -8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    flat = rng.normal(0, 0.3, setnet.NPARAM).astype(np.float32)
    flat = setnet.bf16_round(flat).astype(np.float64)   # already representable
    sets = []
    for _ in range(3):
        n = int(rng.integers(20, 60))
        sets.append((rng.integers(-500, 500, n), rng.integers(-500, 500, n)))
    targets = [(0.3, -0.1), (-0.7, 0.2), (1.1, 0.0)]
    lam = 0.5
    L, g = setnet.loss_and_grad(flat, sets, targets, lam)
    assert abs(L - setnet.loss_only(flat, sets, targets, lam)) < 1e-12
    idx = rng.choice(setnet.NPARAM, 60, replace=False)
    eps = 1e-6
    for k in idx:
        e = np.zeros(setnet.NPARAM)
        e[k] = eps
        num = (setnet.loss_only(flat + e, sets, targets, lam) - setnet.loss_only(flat - e, sets, targets, lam)) / (2 * eps)
        assert abs(num - g[k]) <= 1e-6 + 1e-4 * abs(num), (k, num, g[k])
