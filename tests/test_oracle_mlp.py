"""Pins for the oracle's patch MLP (CPU): backpropagated gradients against central finite
differences, the loss of known networks, and positive homogeneity (no biases, ReLU)."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    din, width, batch = 8, 16, 32
    W = list(mlp.init_weights(din, width, seed=1))
    W[3] = rng.standard_normal((din, din)) * 0.3          # a nonzero skip term
    X = rng.standard_normal((batch, din))
    T = rng.standard_normal((batch, din))
    L, G = mlp.grad(W, X, T)
    h = 1e-6
    for li in range(4):
        for _ in range(12):
            i, j = rng.integers(W[li].shape[0]), rng.integers(W[li].shape[1])
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[li][i, j] += h
            Wm[li][i, j] -= h
            fd = (mlp.loss(Wp, X, T) - mlp.loss(Wm, X, T)) / (2 * h)
            assert abs(fd - G[li][i, j]) <= 1e-6 * max(1.0, abs(fd)), (li, i, j, fd, G[li][i, j])


def test_loss_of_identity_network_is_zero_on_positive_data():
    """W1 = [I, 0], W2 = I, W3 = [I; 0]: y = relu(relu(x)) = x for x >= 0, so L(x, x) = 0."""
    din, width = 5, 9
    W1 = np.zeros((din, width)); W1[:, :din] = np.eye(din)
    W2 = np.eye(width)
    W3 = np.zeros((width, din)); W3[:din, :] = np.eye(din)
    X = np.abs(np.random.default_rng(3).standard_normal((7, din)))
    assert mlp.loss((W1, W2, W3), X, X) == 0.0


def test_skip_only_network_is_linear_least_squares():
    """W1 = W2 = W3 = 0: y = x W0, so L is the relative least-squares residual and its minimiser
    is numpy's lstsq solution, where the gradient vanishes."""
    rng = np.random.default_rng(6)
    din, width = 6, 4
    X = rng.standard_normal((40, din))
    T = rng.standard_normal((40, din))
    W0, *_ = np.linalg.lstsq(X, T, rcond=None)
    Z = (np.zeros((din, width)), np.zeros((width, width)), np.zeros((width, din)))
    L, G = mlp.grad(Z + (W0,), X, T)
    assert abs(L - np.sum((X @ W0 - T) ** 2) / np.sum(T ** 2)) <= 1e-14
    assert np.abs(G[3]).max() <= 1e-12


def test_positive_homogeneity():
    W = list(mlp.init_weights(6, 12, seed=4))
    W[3] = np.random.default_rng(7).standard_normal((6, 6))
    X = np.random.default_rng(5).standard_normal((4, 6))
    Y1, _ = mlp.forward(W, X)
    Y3, _ = mlp.forward(W, 3.0 * X)
    np.testing.assert_allclose(Y3, 3.0 * Y1, rtol=1e-14, atol=1e-14)


def test_width_zero_is_the_linear_map():
    rng = np.random.default_rng(9)
    W = list(mlp.init_weights(5, 0, seed=2))
    assert W[0].shape == (5, 0) and W[1].shape == (0, 0) and W[2].shape == (0, 5)
    W[3] = rng.standard_normal((5, 5))
    X = rng.standard_normal((6, 5))
    Y, _ = mlp.forward(W, X)
    np.testing.assert_array_equal(Y, X @ W[3])
