"""Host-side parts of the variant selection: regret and target definitions,
and the learning set-up itself (features -> relative log-times -> argmin)
trained with the FP64 oracle MLP on the stored GB300 timings, which must beat
the built-in reuse rule on the held-out tensors."""
import os

import numpy as np

from oracle import mlp as omlp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TIMINGS = os.path.join(ROOT, "paper_2102_10245_gb300", "data", "variant_timings.npz")


def _regret(times, picks):
    from paper_2102_10245_gb300.autotune import regret
    return regret(times, picks)


def test_regret_definition():
    t = np.array([[1.0, 2.0, 4.0], [3.0, 1.0, 1.5]])
    assert _regret(t, [0, 1]) == (0.0, 0.0)
    total, mean = _regret(t, [1, 2])
    assert np.isclose(total, (2.0 + 1.5) / (1.0 + 1.0) - 1.0)
    assert np.isclose(mean, (2.0 / 1.0 + 1.5 / 1.0) / 2 - 1.0)


def test_targets_are_log2_ratios():
    from paper_2102_10245_gb300.autotune import targets
    t = np.array([[1.0, 2.0, 4.0], [8.0, 2.0, 2.0]])
    assert np.array_equal(targets(t), [[0.0, 1.0, 2.0], [2.0, 0.0, 0.0]])


def test_learning_setup_beats_rule_on_heldout():
    from paper_2102_10245_gb300.autotune import targets
    d = np.load(TIMINGS)
    X, T = d["train_features"], d["train_times"]
    mu, sd = X.mean(0), X.std(0) + 1e-6
    Xs = (X - mu) / sd
    Y = targets(T)
    rng = np.random.default_rng(0)
    sizes = (X.shape[1], 32, 32, T.shape[1])
    params = [[rng.standard_normal((o, i)) * np.sqrt(2.0 / (i + o)), np.zeros(o)] for i, o in zip(sizes[:-1], sizes[1:])]
    m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    for step in range(1, 401):
        acts = omlp.forward(Xs, params)
        _, dP = omlp.mse(acts[-1], Y)
        grads = omlp.backward(Xs, params, acts, dP)
        for li in range(len(params)):
            for k in range(2):
                params[li][k], m[li][k], v[li][k] = omlp.adam_step(params[li][k], grads[li][k], m[li][k], v[li][k],
                                                                   3e-3, 0.9, 0.999, 1e-8, step)
    H = (d["heldout_features"] - mu) / sd
    picks = omlp.forward(H, params)[-1].argmin(axis=1)
    ht = d["heldout_times"]
    learned = _regret(ht, picks)[0]
    rule = _regret(ht, d["heldout_rule"])[0]
    print("held-out regret: learned %.3f, rule %.3f" % (learned, rule))
    assert learned <= 0.10 and learned < rule
