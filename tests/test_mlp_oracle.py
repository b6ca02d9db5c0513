"""Pins for the cost-network oracle: backpropagated gradients against
central finite differences, and the Adam step against its closed form on
a case whose moments are known."""
import numpy as np

from oracle import mlp as M


def test_backprop_matches_finite_differences():
    F, H, N = 5, 7, 11
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.5, M.param_count(F, H))
    X = rng.normal(0, 1, (N, F))
    T = rng.normal(0, 1, N)
    g = M.grad(p, X, T, F, H)
    idx = list(range(0, M.param_count(F, H), 3))
    num = M.numeric_grad(p, X, T, F, H, idx)
    np.testing.assert_allclose(g[idx], num, rtol=1e-5, atol=1e-8)


def test_forward_special_cases():
    F, H = 3, 4
    p = np.zeros(M.param_count(F, H))
    p[-1] = 2.5                                  # b3 only: constant output
    y, _ = M.forward(p, np.ones((6, F)), F, H)
    assert np.all(y == 2.5)
    # identity-like network on a positive input: y = sum(W3) * relu(W2 relu(W1 x))
    p = np.zeros(M.param_count(F, H))
    W1 = np.zeros((H, F)); W1[0, 0] = 1.0
    W2 = np.zeros((H, H)); W2[0, 0] = 3.0
    o = 0
    p[o:o + H * F] = W1.ravel(); o += H * F + H
    p[o:o + H * H] = W2.ravel(); o += H * H + H
    p[o] = 0.5
    y, _ = M.forward(p, np.array([[2.0, 9.0, 9.0], [-1.0, 0.0, 0.0]]), F, H)
    np.testing.assert_array_equal(y, [3.0, 0.0])   # 0.5 * 3 * 2, and relu kills the negative input


def test_adam_first_step_is_signed_lr():
    # with zero moments, the bias-corrected first step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-6)
