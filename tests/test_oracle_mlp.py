"""Pins for the surrogate-MLP oracle: central finite differences of its float64 form, the
zero-weight network (output = b3), a configuration that reduces to a linear map with a closed
form, and bf16 rounding of exactly representable values (no change) and of a halfway case
(round to even)."""
import numpy as np

import oracle

P = oracle.MLP_PARAMS
W1, B1, W2, B2, W3, B3 = 0, 512, 576, 4672, 4736, 4800


def _rand_params(rng, scale=0.3):
    p = rng.normal(0, scale, P).astype(np.float32)
    p[B1:B1 + 64] = rng.uniform(0.05, 0.3, 64)
    p[B2:B2 + 64] = rng.uniform(0.05, 0.3, 64)
    return p


def test_finite_difference_gradient():
    rng = np.random.default_rng(0)
    p = _rand_params(rng)
    x = rng.normal(0, 1, (37, 8)).astype(np.float32)
    t = rng.normal(0, 1, 37).astype(np.float32)
    g, _ = oracle.mlp_gradient(x, t, p, round_bf16=False)

    def loss(pp):
        y = oracle.mlp_forward(x, pp, round_bf16=False)
        return np.mean((y - t.astype(np.float64)) ** 2)

    idx = np.r_[rng.choice(512, 20, replace=False), B1 + np.arange(0, 64, 7),
                W2 + rng.choice(4096, 30, replace=False), B2 + np.arange(0, 64, 9),
                W3 + np.arange(0, 64, 5), B3]
    h = 1e-5  # small enough that no ReLU pre-activation crosses zero between the two points
    for k in idx:
        a = p.astype(np.float64)
        pp, pm = p.copy(), p.copy()  # the actual float32 step is used in the quotient below
        pp[k] = np.float32(a[k] + h)
        pm[k] = np.float32(a[k] - h)
        fd = (loss(pp) - loss(pm)) / (float(pp[k]) - float(pm[k]))
        assert abs(fd - g[k]) <= 1e-4 * abs(g[k]) + 1e-6, (k, fd, g[k])


def test_zero_weights_give_bias():
    p = np.zeros(P, np.float32)
    p[B3] = 1.25
    x = np.random.default_rng(1).normal(0, 1, (10, 8)).astype(np.float32)
    for r in (True, False):
        assert np.all(oracle.mlp_forward(x, p, round_bf16=r) == 1.25)


def test_linear_regime_closed_form():
    # W1 copies the 8 inputs into units 0..7 with large positive biases keeping every unit
    # active; W2 copies units 0..7 likewise; then y = b3 + sum_k w3_k (x_k + c1 + c2).
    p = np.zeros(P, np.float32)
    for k in range(8):
        p[W1 + k * 64 + k] = 1.0
        p[W2 + k * 64 + k] = 1.0
    p[B1:B1 + 64] = 8.0
    p[B2:B2 + 64] = 4.0
    w3 = np.array([0.5, -1, 2, 0.25, -0.75, 1.5, -2, 1], np.float32)
    p[W3:W3 + 8] = w3
    p[B3] = -3.0
    x = np.random.default_rng(2).integers(-4, 5, (20, 8)).astype(np.float32)
    want = -3.0 + ((x + 12.0) * w3).sum(1)
    np.testing.assert_array_equal(oracle.mlp_forward(x, p, round_bf16=True), want)
    np.testing.assert_array_equal(oracle.mlp_forward(x, p, round_bf16=False), want)


def test_bf16_rounding_points():
    # 1 + 2^-8 is exactly halfway between the bf16 neighbours 1 and 1 + 2^-7: rounds to 1 (even);
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: rounds to 1 + 2^-6.
    p = np.zeros(P, np.float32)
    p[W1 + 0] = 1.0          # unit 0 = x0
    p[W2 + 0] = 1.0          # unit 0 of layer 2 = h1_0
    p[W3 + 0] = 1.0
    x = np.zeros((2, 8), np.float32)
    x[0, 0] = 1 + 2 ** -8
    x[1, 0] = 1 + 3 * 2 ** -8
    y = oracle.mlp_forward(x, p, round_bf16=True)
    assert list(y) == [1.0, 1 + 2 ** -6]
    assert list(oracle.mlp_forward(x, p, round_bf16=False)) == [1 + 2 ** -8, 1 + 3 * 2 ** -8]
