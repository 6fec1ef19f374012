"""The stored autotuner timing set (host-side checks): measured on the current
MTTKRP kernel sources (source hash) for the autotuner's candidates (variant x
segment count), shapes, feature names, finite positive times, the training
and held-out seeds disjoint and those of the batched workload's generator."""
import os

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TIMINGS = os.path.join(ROOT, "paper_2102_10245_gb300", "data", "variant_timings.npz")
FEATURES = (
    "order", "log2_len", "log2_nnz", "log2_reuse", "log2_rank", "distinct_frac", "hot_share",
    "log2_hot_rows", "log2_unit_width_p50", "log2_unit_width_p90", "unit_fit_smem", "log2_max_interval",
    "mean_log2_other_len", "key_words", "log2_gather_bytes",
)


def test_timing_set_shape_and_seeds():
    from paper_2102_10245_gb300 import autotune as tune
    from paper_2102_10245_gb300.build import kernel_source_hash
    d = np.load(TIMINGS)
    # measured on the current MTTKRP kernel sources, with the autotuner's candidates
    assert str(d["kernel_hash"]) == kernel_source_hash()
    assert tuple(d["candidates"]) == tune.VARIANT_LABELS
    for part, seeds in (("train", range(0, 2000)), ("heldout", range(100_000, 100_256))):
        f, t, meta = d[part + "_features"], d[part + "_times"], d[part + "_meta"]
        assert tuple(d[part + "_feature_names"]) == FEATURES
        assert f.shape == (len(t), len(FEATURES)) and t.shape[1] == len(tune.CANDIDATES) and np.isfinite(f).all()
        assert (t > 0).all() and np.isfinite(t).all()
        assert sorted(set(meta[:, 0].tolist())) == list(seeds)
        # every mode of every tensor, with the generator's order and nnz
        for s in list(seeds)[:50]:
            cfg = synth.batch_config(s)
            rows = meta[meta[:, 0] == s]
            assert list(rows[:, 1]) == list(range(len(cfg["dims"])))
            assert (rows[:, 2] == cfg["nnz"]).all()
            assert (f[meta[:, 0] == s][:, 0] == len(cfg["dims"])).all()
