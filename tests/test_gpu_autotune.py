"""The learned variant choice: the autotuner's timing path on live tensors,
the predictor's GPU inference against the FP64 oracle forward with the same
weights, and what the trained predictor gains over the built-in reuse rule
(the method without it) on the held-out batched tensors, judged by the
autotuner's timings (stored in the package's timing set, measured on GB300)."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TIMINGS = os.path.join(ROOT, "paper_2102_10245_gb300", "data", "variant_timings.npz")


@pytest.fixture(scope="module")
def trained(alto_lib):
    from paper_2102_10245_gb300 import autotune as tune
    d = np.load(TIMINGS)
    pred = tune.Predictor(seed=0)
    losses = pred.fit(d["train_features"], d["train_times"], epochs=2000)
    return pred, d, losses


def test_predictor_beats_rule_on_heldout(trained):
    from paper_2102_10245_gb300 import autotune as tune
    pred, d, losses = trained
    assert losses[-1] < 0.5 * losses[0]
    hf, ht, hr = d["heldout_features"], d["heldout_times"], d["heldout_rule"]
    picks = pred.pick(hf)
    mlp_total, mlp_mean = tune.regret(ht, picks)
    rule_total, rule_mean = tune.regret(ht, hr)
    best = ht.min(axis=1).sum()
    print("held-out (%d calls): predictor regret %.3f (mean %.3f), rule %.3f (mean %.3f); "
          "sum of times %.1f ms predictor vs %.1f ms rule vs %.1f ms autotuned"
          % (len(ht), mlp_total, mlp_mean, rule_total, rule_mean, best * (1 + mlp_total), best * (1 + rule_total),
             best))
    assert mlp_total <= 0.10 and mlp_mean <= 0.10
    assert mlp_total < rule_total


def test_autotuner_fallback_never_hurts(trained):
    from paper_2102_10245_gb300 import autotune as tune
    pred, d, _ = trained
    hf, ht = d["heldout_features"], d["heldout_times"]
    pure = tune.regret(ht, pred.pick(hf))[0]
    hybrid = tune.regret(ht, pred.choose(hf, measure=lambda r: ht[r], margin=0.3))[0]
    assert hybrid <= pure + 1e-12


def test_inference_matches_oracle(trained):
    pred, d, _ = trained
    f = d["heldout_features"][:257]
    got = pred.scores(f)
    x = (f - pred.mu) / pred.sd
    params = [[W.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)] for W, b in pred.net.params]
    ref = omlp.forward(x.astype(np.float32), params)[-1]
    assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_live_timing_features_and_rule(alto_lib):
    from paper_2102_10245_gb300 import autotune as tune
    cfg = synth.batch_config(7)
    cfg["dims"] = tuple(min(d, 200_000) for d in cfg["dims"])
    cfg["nnz"] = min(cfg["nnz"], 200_000)
    at, factors = tune.make_item(cfg)
    R = cfg["rank"]
    for n in range(at.N):
        out = torch.empty(at.dims[n], R, device="cuda")
        t = tune.time_variants(at, n, factors, out)
        assert t.shape == (len(tune.VARIANTS),) and np.isfinite(t).all() and (t > 0).all()
        f = tune.features(at, n, R)
        assert f.shape == (len(tune.FEATURES),) and np.isfinite(f).all()
        assert 0 <= tune.rule_pick(at, n, R) < len(tune.VARIANTS)
        # the timing leaves the tensor on the automatic choice and the result exact
        assert at.stats()["variant"][n] == 0
        ref = at.mttkrp(n, factors)
        tune.apply(at, n, int(np.argmin(t)))
        got = at.mttkrp(n, factors)
        torch.cuda.synchronize()
        assert torch.allclose(got, ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))
    at.close()


def test_collect_small(alto_lib):
    from paper_2102_10245_gb300 import autotune as tune
    d = tune.collect([3, 4])
    rows = sum(len(synth.batch_config(s)["dims"]) for s in (3, 4))
    assert d["features"].shape == (rows, len(tune.FEATURES)) and d["times"].shape == (rows, len(tune.VARIANTS))
    assert (d["times"] > 0).all() and list(d["meta"][:, 0]) == [3] * len(synth.batch_config(3)["dims"]) + \
        [4] * len(synth.batch_config(4)["dims"])


def test_configure_save_load(trained, tmp_path):
    from paper_2102_10245_gb300 import autotune as tune
    pred, d, _ = trained
    f = d["heldout_features"][:64]
    path = str(tmp_path / "pred.npz")
    pred.save(path)
    again = tune.Predictor.load(path)
    assert np.array_equal(again.pick(f), pred.pick(f))
    cfg = synth.batch_config(11)
    cfg["dims"] = tuple(min(x, 100_000) for x in cfg["dims"])
    cfg["nnz"] = min(cfg["nnz"], 100_000)
    at, factors = tune.make_item(cfg)
    picks = again.configure(at, cfg["rank"])
    assert at.stats()["variant"] == picks
    at.close()
