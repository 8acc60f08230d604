"""FP64 reference of the patch MLP and its training loss/gradient (oracle; test infrastructure).

The learned preconditioner maps a normalised element-patch residual x (D^3 values) to a
correction y by a three-layer perceptron without biases plus a linear skip term,
    h1 = relu(x W1),  h2 = relu(h1 W2),  y = h2 W3 + x W0,
and is trained on pairs (x, t) by the relative squared error
    L = sum_b ||y_b - t_b||^2 / sum_b ||t_b||^2.
The paper has no learned component; this is the textbook MLP and its backpropagation written
out, pinned by finite differences in tests/test_oracle_mlp.py.  W is (W1, W2, W3, W0); a
3-tuple means W0 = 0; width 0 (empty W1, W2, W3) is the linear patch map y = x W0.
"""
import numpy as np


def relu(z):
    return np.maximum(z, 0.0)


def _weights(W):
    W = [np.asarray(w, dtype=np.float64) for w in W]
    if len(W) == 3:
        W.append(np.zeros((W[0].shape[0], W[2].shape[1])))
    return W


def forward(W, X):
    """W = (W1 [din, w], W2 [w, w], W3 [w, din], W0 [din, din]); X [batch, din].
    Returns (Y, cache)."""
    W1, W2, W3, W0 = _weights(W)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1
    h1 = relu(z1)
    z2 = h1 @ W2
    h2 = relu(z2)
    Y = h2 @ W3 + X @ W0
    return Y, (X, z1, h1, z2, h2)


def loss(W, X, T):
    Y, _ = forward(W, X)
    T = np.asarray(T, dtype=np.float64)
    return float(np.sum((Y - T) ** 2) / np.sum(T ** 2))


def grad(W, X, T):
    """(L, (dW1, dW2, dW3, dW0)) by backpropagation through the three layers and the skip."""
    W1, W2, W3, W0 = _weights(W)
    T = np.asarray(T, dtype=np.float64)
    Y, (X, z1, h1, z2, h2) = forward((W1, W2, W3, W0), X)
    nt = np.sum(T ** 2)
    L = float(np.sum((Y - T) ** 2) / nt)
    dY = 2.0 * (Y - T) / nt
    dW3 = h2.T @ dY
    dW0 = X.T @ dY
    dz2 = (dY @ W3.T) * (z2 > 0)
    dW2 = h1.T @ dz2
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    dW1 = X.T @ dz1
    return L, (dW1, dW2, dW3, dW0)


def init_weights(din, width, seed):
    """He-normal initialisation (std sqrt(2 / fan_in)) of W1, W2, W3, seeded; W0 = 0.  Width 0
    (no hidden layers: the linear map y = x W0) gives empty W1, W2, W3."""
    rng = np.random.default_rng(seed)
    sw = np.sqrt(2.0 / width) if width else 0.0
    return (rng.standard_normal((din, width)) * np.sqrt(2.0 / din),
            rng.standard_normal((width, width)) * sw,
            rng.standard_normal((width, din)) * sw,
            np.zeros((din, din)))
