"""The variant-predictor MLP on the GPU: parameters live in device tensors,
every forward, backward, loss and Adam step is one of libalto's nn kernels
(``alto_nn_*``); this module only sequences the calls."""
import ctypes

import torch

from .alto import _check, _stream, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class MLP:
    """Fully connected network din -> hidden... -> dout, ReLU between layers."""

    def __init__(self, sizes, seed=0, device="cuda"):
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.sizes = list(sizes)
        self.params = []
        for din, dout in zip(sizes[:-1], sizes[1:]):
            bound = (6.0 / (din + dout)) ** 0.5
            W = ((torch.rand(dout, din, generator=g) * 2 - 1) * bound).to(device).contiguous()
            b = torch.zeros(dout, device=device)
            self.params.append([W, b])
        self.m = [[torch.zeros_like(W), torch.zeros_like(b)] for W, b in self.params]
        self.v = [[torch.zeros_like(W), torch.zeros_like(b)] for W, b in self.params]
        self.step = 0
        self.device = device

    def forward(self, X, stream=None):
        """List of every layer's output (post-activation)."""
        X = X.contiguous()
        acts = []
        h = X
        n = X.shape[0]
        for li, (W, b) in enumerate(self.params):
            Y = torch.empty(n, W.shape[0], device=self.device)
            relu = 1 if li + 1 < len(self.params) else 0
            _check(lib().alto_nn_linear_forward(_p(h), _p(W), _p(b), _p(Y), n, W.shape[1], W.shape[0], relu,
                                                _stream(stream)))
            acts.append(Y)
            h = Y
        return acts

    def predict(self, X):
        return self.forward(X)[-1]

    def loss_and_grads(self, X, T, mask=None, stream=None):
        acts = self.forward(X, stream)
        P = acts[-1]
        n = X.shape[0]
        dP = torch.empty_like(P)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        norm = float(mask.sum().item()) if mask is not None else float(P.numel())
        _check(lib().alto_nn_mse(_p(P), _p(T.contiguous()), _p(mask), _p(dP), P.numel(), norm, _p(loss),
                                 _stream(stream)))
        grads = [None] * len(self.params)
        dY = dP
        for li in range(len(self.params) - 1, -1, -1):
            W, b = self.params[li]
            h_in = X if li == 0 else acts[li - 1]
            G = torch.empty_like(acts[li])
            dW = torch.empty_like(W)
            db = torch.empty_like(b)
            dX = torch.empty(n, W.shape[1], device=self.device) if li > 0 else None
            relu = 1 if li + 1 < len(self.params) else 0
            _check(lib().alto_nn_linear_backward(_p(h_in), _p(W), _p(acts[li]), _p(dY), _p(G), _p(dX), _p(dW), _p(db),
                                                 n, W.shape[1], W.shape[0], relu, _stream(stream)))
            grads[li] = (dW, db)
            dY = dX
        return loss, grads

    def adam(self, grads, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        self.step += 1
        for li, (dW, db) in enumerate(grads):
            for k, g in enumerate((dW, db)):
                p = self.params[li][k]
                _check(lib().alto_nn_adam(_p(p), _p(g), _p(self.m[li][k]), _p(self.v[li][k]), p.numel(), lr, b1, b2,
                                          eps, self.step, _stream(stream)))

    def fit(self, X, T, mask=None, epochs=2000, lr=1e-3):
        losses = []
        for e in range(epochs):
            loss, grads = self.loss_and_grads(X, T, mask)
            self.adam(grads, lr=lr)
            if e % 100 == 0 or e == epochs - 1:
                losses.append(float(loss.item()))
        return losses

    def state(self):
        return [[W.cpu().numpy(), b.cpu().numpy()] for W, b in self.params]
