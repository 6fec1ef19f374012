"""Full-size workloads, in the launch configuration bench.py times (library
defaults: automatic variant, default segments).  Outputs are checked on
sampled rows the oracle computes one by one, and the format by properties
that hold at any size plus sampled recomputation."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import dev, dev_idx, rel_err, to_bf16_exact

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_CACHE = {}


def _tensor(name):
    if name not in _CACHE:
        _CACHE.clear()
        cfg = synth.CONFIGS[name]
        dims, idx, vals = synth.tensor(cfg)
        _CACHE[name] = (cfg, dims, idx, vals)
    return _CACHE[name]


def _sample_rows(rng, I, k=10_000):
    return np.unique(rng.integers(0, I, k)) if I > k else np.arange(I)


def _check_format_sampled(dims, idx, vals, at):
    ex = at.export()
    lay = at.layout()
    st = at.stats()
    M = len(vals)
    kw = lay["key_words"]
    keys = ex["keys"].copy()
    for b in list(lay["flag_bit"]) + list(lay["hot_bit"]):
        if b >= 0:
            keys[:, b // 64] &= ~np.uint64(1 << (b % 64))
    # ascending keys; perm a permutation; sampled keys equal the oracle encode
    if kw == 1:
        assert (keys[1:, 0] >= keys[:-1, 0]).all()
    else:
        hi, lo = keys[:, 1], keys[:, 0]
        assert ((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] >= lo[:-1]))).all()
    perm = ex["perm"].astype(np.int64)
    assert (np.bincount(perm, minlength=M) == 1).all()
    rng = np.random.default_rng(0)
    pos = rng.integers(0, M, 100_000)
    src = perm[pos]
    ok = oracle.encode(dims, [a[src] for a in idx])
    assert (keys[pos] == ok[:, :kw]).all()
    assert (ex["vals"][pos] == vals[src]).all()
    # intervals of sampled segments, distinct counts
    b = ex["bounds"]
    for l in rng.integers(0, len(b) - 1, 200):
        seg = oracle.decode(dims, np.concatenate([keys[b[l]:b[l + 1]], np.zeros((b[l + 1] - b[l], 2 - kw), np.uint64)], 1))
        assert (ex["intervals"][l, :, 0] == seg.min(0)).all() and (ex["intervals"][l, :, 1] == seg.max(0)).all()
    for n in range(len(dims)):
        assert st["distinct"][n] == int((np.bincount(idx[n], minlength=dims[n]) > 0).sum())


def _mttkrp_sampled(at, dims, idx, vals, U, Ud, label, tol, U_ref=None):
    rng = np.random.default_rng(1)
    worst = 0.0
    for n in range(len(dims)):
        rows = _sample_rows(rng, dims[n])
        got = at.mttkrp(n, Ud).cpu().numpy()[rows]
        ref = oracle.mttkrp(dims, idx, vals, U_ref if U_ref is not None else U, n, rows=rows)[rows]
        e = rel_err(got, ref)
        worst = max(worst, e)
        print("%s mode %d: rel err %.3e on %d sampled rows (variant %d)" % (label, n, e, len(rows), at.stats()["variant"][n]))
        assert e <= tol, (label, n, e)
    return worst


def test_zipf3d_full_fp32():
    cfg, dims, idx, vals = _tensor("zipf3d-4Mx4Mx30k")
    U = synth.factors(cfg)
    from paper_2102_10245_gb300 import AltoTensor
    at = AltoTensor(dims, dev_idx(idx), dev(vals))
    _check_format_sampled(dims, idx, vals, at)
    Ud = [dev(u) for u in U]
    _mttkrp_sampled(at, dims, idx, vals, U, Ud, "zipf3d fp32", 1e-5)
    # CP-ALS at full size: the fit never decreases (ALS monotonicity)
    lam, fits = at.cpals([dev(u.copy()) for u in U], 4)
    print("zipf3d fits", fits)
    assert all(b >= a - 1e-6 for a, b in zip(fits, fits[1:]))


def test_long5d_full_fp32_and_bf16():
    cfg, dims, idx, vals = _tensor("long5d-2^20x3-2^16x2")
    U = synth.factors(cfg)
    from paper_2102_10245_gb300 import AltoTensor
    at = AltoTensor(dims, dev_idx(idx), dev(vals))
    assert at.layout()["key_words"] == 2
    _check_format_sampled(dims, idx, vals, at)
    _mttkrp_sampled(at, dims, idx, vals, U, [dev(u) for u in U], "long5d fp32", 1e-5)
    pairs = [to_bf16_exact(u) for u in U]
    _mttkrp_sampled(at, dims, idx, vals, U, [p[0] for p in pairs], "long5d bf16 (vs fp32 factors)", 1e-2)


def test_clustered4d_full_bf16_vs_fp32():
    cfg, dims, idx, vals = _tensor("clustered4d-12kx60kx5Mx100")
    U = synth.factors(cfg)
    from paper_2102_10245_gb300 import AltoTensor
    at = AltoTensor(dims, dev_idx(idx), dev(vals))
    e32 = _mttkrp_sampled(at, dims, idx, vals, U, [dev(u) for u in U], "clustered4d fp32", 1e-5)
    pairs = [to_bf16_exact(u) for u in U]
    eb = _mttkrp_sampled(at, dims, idx, vals, U, [p[0] for p in pairs], "clustered4d bf16 (vs fp32 factors)", 1e-2)
    er = _mttkrp_sampled(at, dims, idx, vals, U, [p[0] for p in pairs], "clustered4d bf16 (vs rounded)", 1e-5,
                         U_ref=[p[1] for p in pairs])
    print("clustered4d: FP32 %.2e, BF16 %.2e vs FP64 oracle; BF16 accumulation %.2e" % (e32, eb, er))
