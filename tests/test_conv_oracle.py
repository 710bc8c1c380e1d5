"""Pins of the CPU convolution oracle: closed forms (identity and shift kernels) and finite
differences of its gradients."""
import numpy as np

from oracle import conv_oracle as CO


def test_identity_and_shift_kernels():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 7, 3))
    w = np.zeros((3, 3, 3, 3))
    w[:, 1, 1, :] = np.eye(3)
    np.testing.assert_allclose(CO.conv3x3(x, w), x, atol=1e-15)
    w = np.zeros((3, 3, 3, 3))
    w[:, 0, 2, :] = np.eye(3)  # tap (dy, dx) = (-1, +1): y[i, j] = x[i - 1, j + 1]
    y = CO.conv3x3(x, w)
    np.testing.assert_allclose(y[2, 3], x[1, 4], atol=1e-15)
    np.testing.assert_allclose(y[0, 6], x[4, 0], atol=1e-15)  # periodic wrap in both directions


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 6, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    G = rng.normal(size=(4, 6, 2))  # L = sum G * y
    dx = CO.conv3x3_grad_input(G, w)
    dw, db = CO.conv3x3_grad_weight(x, G)
    h = 1e-6
    L = lambda xx, ww, bb: np.sum(G * CO.conv3x3(xx, ww, bb))  # noqa: E731
    for idx in [(0, 0, 0), (3, 5, 2), (1, 2, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert abs((L(x + e, w, b) - L(x - e, w, b)) / (2 * h) - dx[idx]) < 1e-7
    for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (0, 1, 2, 1)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert abs((L(x, w + e, b) - L(x, w - e, b)) / (2 * h) - dw[idx]) < 1e-7
    e = np.array([h, 0.0])
    assert abs((L(x, w, b + e) - L(x, w, b - e)) / (2 * h) - db[0]) < 1e-7


def test_bf16_rounding_is_round_to_nearest_even():
    assert CO.bf16_round(1.0 + 2 ** -8) == 1.0          # tie -> even
    assert CO.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert CO.bf16_round(1.0 + 2 ** -7) == 1.0 + 2 ** -7
