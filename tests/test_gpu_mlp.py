"""The variant predictor's CUDA kernels (dense forward with ReLU, backward,
masked MSE, Adam) against the FP64 oracle on ragged shapes, and a short
training run whose loss falls."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


@pytest.mark.parametrize("n", [1, 37, 1000, 4099])
@pytest.mark.parametrize("sizes", [(15, 64, 64, 3), (3, 1, 5), (9, 33, 2)])
def test_forward_backward_against_oracle(alto_lib, n, sizes):
    from paper_2102_10245_gb300.mlp import MLP
    rng = np.random.default_rng(n + len(sizes))
    net = MLP(sizes, seed=n)
    X = rng.standard_normal((n, sizes[0])).astype(np.float32)
    T = rng.standard_normal((n, sizes[-1])).astype(np.float32)
    mask = (rng.random((n, sizes[-1])) * 2).astype(np.float32)
    params = [[W.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)] for W, b in net.params]
    Xd = torch.from_numpy(X).cuda()
    acts = net.forward(Xd)
    ref = omlp.forward(X, params)
    for a, r in zip(acts, ref):
        assert _rel(a.cpu().numpy(), r) <= 1e-5
    norm = float(mask.sum())
    loss, grads = net.loss_and_grads(Xd, torch.from_numpy(T).cuda(), torch.from_numpy(mask).cuda())
    rloss, dP = omlp.mse(ref[-1], T, mask, norm)
    assert abs(loss.item() - rloss) <= 1e-5 * max(rloss, 1e-30)
    rgrads = omlp.backward(X, params, ref, dP)
    for (dW, db), (rW, rb) in zip(grads, rgrads):
        assert _rel(dW.cpu().numpy(), rW) <= 1e-4
        assert _rel(db.cpu().numpy(), rb) <= 1e-4


def test_input_gradient_kernel(alto_lib):
    """dX of the first hidden layer, through the C ABI directly."""
    import ctypes
    from paper_2102_10245_gb300.alto import lib
    rng = np.random.default_rng(7)
    n, din, dout = 53, 10, 17
    X = rng.standard_normal((n, din)).astype(np.float32)
    W = rng.standard_normal((dout, din)).astype(np.float32)
    b = rng.standard_normal(dout).astype(np.float32)
    dY = rng.standard_normal((n, dout)).astype(np.float32)
    d = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    Xd, Wd, bd, dYd = d(X), d(W), d(b), d(dY)
    Y = torch.empty(n, dout, device="cuda")
    G, dX = torch.empty_like(Y), torch.empty(n, din, device="cuda")
    dW, db = torch.empty_like(Wd), torch.empty_like(bd)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib().alto_nn_linear_forward(p(Xd), p(Wd), p(bd), p(Y), n, din, dout, 1, s) == 0
    assert lib().alto_nn_linear_backward(p(Xd), p(Wd), p(Y), p(dYd), p(G), p(dX), p(dW), p(db), n, din, dout, 1, s) == 0
    torch.cuda.synchronize()
    Z = X.astype(np.float64) @ W.T.astype(np.float64) + b
    Gr = dY * (Z > 0)
    assert _rel(dX.cpu().numpy(), Gr @ W.astype(np.float64)) <= 1e-5
    assert _rel(dW.cpu().numpy(), Gr.T @ X.astype(np.float64)) <= 1e-5
    assert _rel(db.cpu().numpy(), Gr.sum(0)) <= 1e-5


def test_adam_against_oracle(alto_lib):
    from paper_2102_10245_gb300.mlp import MLP
    net = MLP((4, 8, 2), seed=1)
    rng = np.random.default_rng(2)
    ref = [[W.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)] for W, b in net.params]
    m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in ref]
    v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in ref]
    for step in range(1, 6):
        grads = [(rng.standard_normal(W.shape).astype(np.float32), rng.standard_normal(b.shape).astype(np.float32))
                 for W, b in ref]
        net.adam([(torch.from_numpy(a).cuda(), torch.from_numpy(c).cuda()) for a, c in grads], lr=0.01)
        for li in range(len(ref)):
            for k in range(2):
                ref[li][k], m[li][k], v[li][k] = omlp.adam_step(ref[li][k], grads[li][k].astype(np.float64),
                                                                m[li][k], v[li][k], 0.01, 0.9, 0.999, 1e-8, step)
    for (W, b), (rW, rb) in zip(net.params, ref):
        assert np.abs(W.cpu().numpy() - rW).max() <= 1e-5
        assert np.abs(b.cpu().numpy() - rb).max() <= 1e-5


def test_training_reduces_loss(alto_lib):
    from paper_2102_10245_gb300.mlp import MLP
    rng = np.random.default_rng(11)
    X = rng.standard_normal((512, 6)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]) + X[:, 1] ** 2, np.abs(X[:, 2]) - X[:, 3]], 1).astype(np.float32)
    net = MLP((6, 32, 32, 2), seed=3)
    losses = net.fit(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), epochs=800, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0], losses
