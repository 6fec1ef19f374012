"""Seeded synthetic inputs: deterministic, distinct, in range, and shaped
as the configuration says."""
import numpy as np

import synth


def _check(cfg):
    d1, i1, v1 = synth.tensor(cfg)
    d2, i2, v2 = synth.tensor(cfg)
    assert all((a == b).all() for a, b in zip(i1, i2)) and (v1 == v2).all()
    M = cfg["nnz"]
    assert len(v1) == M and all(len(a) == M for a in i1)
    for a, d in zip(i1, d1):
        assert a.dtype == np.uint32 and int(a.max()) < d
    c = np.stack([a.astype(np.int64) for a in i1], 1)
    assert len(np.unique(c, axis=0)) == M
    return d1, i1, v1


def test_uniform_small_config():
    d, idx, v = _check(synth.CONFIGS["uniform3d-64x128x256"])
    assert d == (64, 128, 256) and v.dtype == np.float64 and (v >= 0).all() and (v < 1).all()


def test_zipf_scaled_is_skewed():
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=200_000)
    d, idx, v = _check(cfg)
    counts = np.bincount(idx[2], minlength=d[2])
    top = np.sort(counts)[::-1]
    assert top[0] > 50 * np.median(counts[counts > 0])   # heavy head
    assert v.dtype == np.float32 and (v > 0).all()


def test_clustered_and_long_index_scaled():
    _check(synth.scaled("clustered4d-12kx60kx5Mx100", nnz=100_000))
    d, idx, v = _check(synth.scaled("long5d-2^20x3-2^16x2", nnz=100_000))
    assert len(d) == 5


def test_saturated_topup():
    # 95% of all cells: the draw must top up many times and still end distinct
    cfg = dict(dims=(10, 10, 10), nnz=950, laws=(("zipf", 1.5),) * 3, vals="uniform01",
               vdtype="f32", rank=4, fdist="normal", fdtype="f32", iters=1, seed=9)
    _check(cfg)


def test_batch_configs():
    for s in range(5):
        cfg = synth.batch_config(s)
        assert 3 <= len(cfg["dims"]) <= 5 and cfg["rank"] in (8, 16, 32, 64)
        cfg["nnz"] = min(cfg["nnz"], 20_000)
        _check(cfg)


def test_factors_dtype_and_shape():
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    f = synth.factors(cfg)
    assert [x.shape for x in f] == [(64, 16), (128, 16), (256, 16)]
    assert all(x.dtype == np.float64 for x in f)


def test_torch_generator_draws_distinct_in_range_coordinates():
    """The device-side generator (run here on the CPU): exact nnz, indices
    inside their modes, no duplicate coordinate, values in [0, 1), factors
    of the configured shape; Zipf modes skewed toward few rows."""
    import numpy as np
    import torch
    for seed in (0, 1, 2, 5, 9):
        cfg = dict(synth.batch_config(seed))
        cfg["nnz"] = min(cfg["nnz"], 50_000)
        dims, idx, vals = synth.tensor_torch(cfg, "cpu")
        M = cfg["nnz"]
        assert len(vals) == M and all(len(a) == M for a in idx)
        coords = np.stack([a.numpy().astype(np.int64) for a in idx], 1)
        assert (coords >= 0).all() and (coords < np.array(dims)).all()
        assert len(np.unique(coords, axis=0)) == M
        assert float(vals.min()) >= 0.0 and float(vals.max()) < 1.0
        U = synth.factors_torch(cfg, "cpu", torch.bfloat16)
        assert [tuple(u.shape) for u in U] == [(d, cfg["rank"]) for d in dims]
        assert all(u.dtype == torch.bfloat16 for u in U)
        if cfg["laws"][0] not in ("uniform", "clustered"):
            n = int(np.argmax(dims))
            counts = np.bincount(coords[:, n], minlength=dims[n])
            top = np.sort(counts)[::-1][: max(1, dims[n] // 100)].sum()
            assert top > 0.05 * M     # the top 1% of rows hold a visible share
