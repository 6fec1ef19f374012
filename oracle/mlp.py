"""Plain FP64 reference of the variant-predictor MLP (test infrastructure).

Dense layers y = act(x W^T + b) with ReLU on the hidden layers, a masked
mean-squared-error loss and Adam, written from their textbook definitions;
the tests check the CUDA kernels' outputs and gradients against these and
check these gradients against finite differences.
"""
import numpy as np


def forward(X, params):
    """params: list of (W, b); ReLU after every layer but the last.
    Returns the list of layer outputs (post-activation)."""
    acts = []
    h = np.asarray(X, dtype=np.float64)
    for li, (W, b) in enumerate(params):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        h = np.maximum(z, 0.0) if li + 1 < len(params) else z
        acts.append(h)
    return acts


def mse(P, T, mask=None, norm=None):
    """loss = sum(mask (P - T)^2) / norm and its gradient with respect to P."""
    P = np.asarray(P, np.float64)
    T = np.asarray(T, np.float64)
    m = np.ones_like(P) if mask is None else np.asarray(mask, np.float64)
    norm = float(m.sum()) if norm is None else float(norm)
    d = P - T
    return float((m * d * d).sum() / norm), 2.0 * m * d / norm


def backward(X, params, acts, dY):
    """Gradients (dW, db) of every layer given dLoss/dOutput."""
    grads = [None] * len(params)
    g = np.asarray(dY, np.float64)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        if li + 1 < len(params):
            g = g * (acts[li] > 0.0)
        h_in = np.asarray(X, np.float64) if li == 0 else acts[li - 1]
        grads[li] = (g.T @ h_in, g.sum(axis=0))
        g = g @ np.asarray(W, np.float64)
    return grads


def loss_of(X, params, T, mask=None, norm=None):
    return mse(forward(X, params)[-1], T, mask, norm)[0]


def adam_step(p, g, m, v, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return p, m, v
