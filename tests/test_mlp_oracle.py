"""The FP64 MLP oracle pinned to what the mathematics fixes: gradients by
central finite differences, the loss of a known case, ReLU masking, and the
first Adam step's closed form (m_hat = g, v_hat = g^2, so the step is
lr * g / (|g| + eps))."""
import numpy as np

from oracle import mlp


def _net(sizes, seed):
    rng = np.random.default_rng(seed)
    return [[rng.standard_normal((o, i)) * 0.7, rng.standard_normal(o) * 0.3] for i, o in zip(sizes[:-1], sizes[1:])]


def test_mse_known_case():
    P = np.array([[1.0, 2.0], [3.0, 5.0]])
    T = np.array([[0.0, 2.0], [1.0, 1.0]])
    loss, dP = mlp.mse(P, T)
    assert loss == (1 + 0 + 4 + 16) / 4
    assert np.array_equal(dP, 2 * (P - T) / 4)
    mask = np.array([[1.0, 0.0], [0.0, 2.0]])
    loss, dP = mlp.mse(P, T, mask, norm=3.0)
    assert loss == (1 + 2 * 16) / 3
    assert np.array_equal(dP, 2 * mask * (P - T) / 3)


def test_forward_relu_and_linear_output():
    params = [[np.array([[1.0, -1.0], [-2.0, 0.5]]), np.array([0.0, 1.0])], [np.array([[1.0, 1.0]]), np.array([0.5])]]
    X = np.array([[1.0, 2.0], [3.0, -1.0]])
    acts = mlp.forward(X, params)
    # layer 1: row 0 -> (-1, -1) -> relu (0, 0); row 1 -> (4, -5.5) -> (4, 0)
    assert np.array_equal(acts[0], [[0.0, 0.0], [4.0, 0.0]])
    assert np.array_equal(acts[1], [[0.5], [4.5]])
    # no ReLU on the last layer: a negative output stays negative
    params[1][1] = np.array([-10.0])
    assert mlp.forward(X, params)[1][0, 0] == -10.0


def test_gradients_against_finite_differences():
    rng = np.random.default_rng(3)
    sizes = (5, 7, 6, 3)
    params = _net(sizes, 1)
    X = rng.standard_normal((11, 5))
    T = rng.standard_normal((11, 3))
    mask = rng.random((11, 3)) * 2
    acts = mlp.forward(X, params)
    _, dP = mlp.mse(acts[-1], T, mask, norm=7.0)
    grads = mlp.backward(X, params, acts, dP)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            for j in range(0, flat.size, max(1, flat.size // 9)):
                old = flat[j]
                flat[j] = old + h
                lp = mlp.loss_of(X, params, T, mask, 7.0)
                flat[j] = old - h
                lm = mlp.loss_of(X, params, T, mask, 7.0)
                flat[j] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g.reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (li, j, fd, g.reshape(-1)[j])


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    lr, eps = 0.01, 1e-8
    q, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), lr, 0.9, 0.999, eps, 1)
    assert np.allclose(q, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a zero gradient leaves the parameter alone
    q, _, _ = mlp.adam_step(p, np.zeros(3), np.zeros(3), np.zeros(3), lr, 0.9, 0.999, eps, 1)
    assert np.array_equal(q, p)
