"""The set-network oracle's backward pass equals finite differences of its
loss (float64); bf16 rounding matches the IEEE round-to-nearest-even rule;
a sparse network's forward pass and the set frame match values worked out
by hand (ReLUs, max-pooling, biases, the bounding-box frame and the target
definition)."""
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


def _pack(P):
    return np.concatenate([P[name].ravel() for name, _ in setnet.SHAPES])


def test_forward_by_hand():
    # a sparse network whose outputs follow by hand: frame of
    # x = {0, 10, 4}, y = {0, 4, 2} is centre (5, 2), scale 5, so the
    # normalised points are xn = (-1, 1, -0.2), yn = (-0.4, 0.4, 0)
    P = {name: np.zeros(shp) for name, shp in setnet.SHAPES}
    P["W1"][0, 0] = 1.0     # h1_0 = relu(xn)   -> pooled max 1
    P["W1"][1, 0] = -1.0    # h1_1 = relu(-xn)  -> pooled max 1
    P["W1"][2, 1] = 1.0     # h1_2 = relu(yn)   -> pooled max 0.4
    P["b1"][3] = -2.0       # h1_3 = relu(-2) = 0 everywhere
    for c in range(4):
        P["W2"][c, c] = 1.0
    P["W2"][4, 3] = 1.0
    P["b2"][4] = 0.5        # h2_4 = relu(h1_3 + 0.5) = 0.5
    P["W3"][0, 0] = 1.0     # h3_0 = 1
    P["W3"][1, 1] = -1.0    # h3_1 = relu(-1) = 0
    P["W3"][2, 2] = 1.0     # h3_2 = 0.4
    P["W3"][3, 4] = 2.0     # h3_3 = 1
    P["W4"][0, 0] = 2.0
    P["W4"][0, 1] = 5.0     # multiplies the clipped unit: contributes 0
    P["W4"][0, 3] = 0.25
    P["W4"][1, 2] = 1.0
    P["b4"][:] = (0.5, -1.0)
    x, y = [0, 10, 4], [0, 4, 2]
    assert setnet.frame(x, y) == (5.0, 2.0, 5.0)
    phi, b, _ = setnet.forward(_pack(P), x, y)
    assert abs(phi - (2.0 * 1.0 + 0.25 * 1.0 + 0.5)) < 1e-12
    assert abs(b - (0.4 - 1.0)) < 1e-12
    # the loss of the same parameters (no rounding needed: all exact in bf16)
    L = setnet.loss_only(_pack(P), [(x, y)], [(2.0, 0.0)], 0.5)
    assert abs(L - ((phi - 2.0) ** 2 + 0.5 * b * b)) < 1e-12


def test_frame_scale_floor_and_target_definition():
    # scale is half the larger side, at least 1; a single point has scale 1
    assert setnet.frame([3, 3], [7, 8]) == (3.0, 7.5, 1.0)
    assert setnet.frame([0, 40], [0, 10]) == (20.0, 5.0, 20.0)
    # target of the line y = x through a frame centred at (20, 5), scale 20:
    # angle pi/4, normalised intercept (0 - 5 + 1 * 20) / 20
    phi, bn = setnet.targets_from_fit([0, 40], [0, 10], 1.0, 0.0)
    assert abs(phi - np.pi / 4) < 1e-15 and abs(bn - 0.75) < 1e-15
