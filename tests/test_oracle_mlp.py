"""Pins of the oracle's proposer MLP (forward, binary cross-entropy, backprop).

The gradient is checked against central finite differences of the loss, the
loss against its closed form at zero weights, and GELU against Phi values."""
import numpy as np

import oracle


def _params(rng, m, h1, h2, K, scale=0.5):
    offs = oracle.mlp_sizes(m, h1, h2, K)
    return rng.standard_normal(offs[-1]) * scale, offs


def test_loss_at_zero_weights_is_K_log2():
    m, h1, h2, K = 4, 5, 3, 7
    offs = oracle.mlp_sizes(m, h1, h2, K)
    p = np.zeros(offs[-1])
    Y = np.random.default_rng(0).standard_normal((9, m))
    idx = np.array([[0, 3], [1, -1], [6, 2]] * 3, np.int32)
    loss, g = oracle.mlp_loss_grad(p, m, h1, h2, K, Y, idx)
    assert abs(loss - K * np.log(2.0)) < 1e-14
    # only the output bias sees a gradient: (sigmoid(0) - t) / B summed over the batch
    t = np.zeros((9, K))
    for b in range(9):
        for j in idx[b]:
            if j >= 0:
                t[b, j] = 1
    np.testing.assert_allclose(g[offs[5]:offs[6]], (0.5 - t).sum(axis=0) / 9, atol=1e-15)
    assert np.abs(g[:offs[5]]).max() == 0


def test_gelu_values_through_a_one_unit_network():
    """m=1, h1=h2=1, K=1 with unit weights and zero biases: z = gelu(gelu(y)) with
    gelu(x) = x Phi(x); Phi from scipy's normal distribution."""
    from scipy.stats import norm
    offs = oracle.mlp_sizes(1, 1, 1, 1)
    p = np.zeros(offs[-1])
    p[offs[0]] = p[offs[2]] = p[offs[4]] = 1.0
    for y in (-2.0, -0.3, 0.0, 1.0, 2.5):
        g1 = y * norm.cdf(y)
        z = oracle.mlp_forward(p, 1, 1, 1, 1, np.array([[y]]))[0, 0]
        assert abs(z - g1 * norm.cdf(g1)) < 1e-13


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    m, h1, h2, K, B = 5, 7, 6, 8, 4
    p, offs = _params(rng, m, h1, h2, K)
    Y = rng.standard_normal((B, m))
    idx = np.array([[1, 4], [0, -1], [7, 2], [3, 5]], np.int32)
    loss, g = oracle.mlp_loss_grad(p, m, h1, h2, K, Y, idx)
    h = 1e-6
    num = np.empty_like(p)
    for q in range(len(p)):
        e = np.zeros_like(p)
        e[q] = h
        lp, _ = oracle.mlp_loss_grad(p + e, m, h1, h2, K, Y, idx, with_grad=False)
        lm, _ = oracle.mlp_loss_grad(p - e, m, h1, h2, K, Y, idx, with_grad=False)
        num[q] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_forward_matches_loss_definition():
    rng = np.random.default_rng(2)
    m, h1, h2, K, B = 6, 8, 5, 10, 5
    p, offs = _params(rng, m, h1, h2, K)
    Y = rng.standard_normal((B, m))
    idx = rng.integers(0, K, size=(B, 3)).astype(np.int32)
    z = oracle.mlp_forward(p, m, h1, h2, K, Y)
    t = np.zeros((B, K))
    for b in range(B):
        t[b, idx[b]] = 1
    want = (np.maximum(z, 0) - z * t + np.log1p(np.exp(-np.abs(z)))).sum() / B
    loss, _ = oracle.mlp_loss_grad(p, m, h1, h2, K, Y, idx, with_grad=False)
    assert abs(loss - want) < 1e-12
