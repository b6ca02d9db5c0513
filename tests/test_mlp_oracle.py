"""Pins for the cost-network oracle: backpropagated gradients against
central finite differences, the forward pass on networks whose output is
known, and the Adam step on cases whose moments are known.  Planted
mistakes in the oracle (on the CPU) must each fail one of these pins."""
import numpy as np
import pytest

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
    # a negative second-layer weight: the second relu clamps W2 relu(W1 x) = -6 to 0
    p[H * F + H] = -3.0
    y, _ = M.forward(p, np.array([[2.0, 9.0, 9.0]]), F, H)
    np.testing.assert_array_equal(y, [0.0])


def test_adam_first_step_is_signed_lr():
    # with zero moments, the bias-corrected first step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-6)


def test_adam_constant_gradient_steps():
    # with the same gradient every step the bias-corrected moments are g and
    # g^2 exactly, so every step moves by lr * g / (|g| + eps)
    g = np.array([0.5, -4.0])
    p, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for step in range(1, 6):
        q, m, v = M.adam_step(p, g, m, v, step, 0.01)
        np.testing.assert_allclose(q - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        p = q


# ---------------------------------------------------------------- planted mistakes

_forward, _grad, _adam = M.forward, M.grad, M.adam_step


def _mut_grad_mask_wrong_layer(p, X, T, F, H):
    W1, b1, W2, b2, W3, b3 = M.unpack(p, F, H)
    X, T = np.asarray(X, dtype=np.float64), np.asarray(T, dtype=np.float64)
    y, (z1, h1, z2, h2) = M.forward(p, X, F, H)
    dy = 2.0 * (y - T) / X.shape[0]
    dh2 = np.outer(dy, W3[0]) * (z1 > 0)          # the first layer's mask
    dh1 = (dh2 @ W2) * (z1 > 0)
    return np.concatenate([(dh1.T @ X).ravel(), dh1.sum(axis=0), (dh2.T @ h1).ravel(), dh2.sum(axis=0),
                           dy @ h2, [dy.sum()]])


def _mut_grad_half(p, X, T, F, H):
    return 0.5 * _grad(p, X, T, F, H)             # the loss derivative without its factor 2


def _mut_forward_second_relu_dropped(p, X, F, H):
    W1, b1, W2, b2, W3, b3 = M.unpack(p, F, H)
    z1 = np.asarray(X, dtype=np.float64) @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    return (z2 @ W3.T + b3)[:, 0], (z1, h1, z2, z2)


def _mut_forward_no_output_bias(p, X, F, H):
    y, acts = _forward(p, X, F, H)
    return y - M.unpack(p, F, H)[5][0], acts


def _mut_adam_no_bias_correction(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    return p - lr * m / (np.sqrt(v) + eps), m, v


def _mut_adam_correction_frozen(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    return _adam(p, g, m, v, 1, lr, b1, b2, eps)   # the first step's correction forever


MLP_MUTANTS = {
    "grad_relu_mask_of_first_layer": ("grad", _mut_grad_mask_wrong_layer),
    "grad_missing_factor_two": ("grad", _mut_grad_half),
    "forward_second_relu_dropped": ("forward", _mut_forward_second_relu_dropped),
    "forward_output_bias_ignored": ("forward", _mut_forward_no_output_bias),
    "adam_without_bias_correction": ("adam_step", _mut_adam_no_bias_correction),
    "adam_bias_correction_frozen": ("adam_step", _mut_adam_correction_frozen),
}

MLP_PINS = [test_backprop_matches_finite_differences, test_forward_special_cases,
            test_adam_first_step_is_signed_lr, test_adam_constant_gradient_steps]


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_planted_mistake_in_network_oracle_is_caught(monkeypatch, name):
    attr, fn = MLP_MUTANTS[name]
    monkeypatch.setattr(M, attr, fn)
    caught = 0
    for pin in MLP_PINS:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake {name}"
