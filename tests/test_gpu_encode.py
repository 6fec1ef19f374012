"""ALTO generation on the GPU (linearization, ordering, value permutation,
partitioning, intervals, distinct counts, helper flags) against the oracle,
bit-exact (Sec. 3.1-3.3)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import dev, dev_idx, make, oracle_format

pytestmark = pytest.mark.gpu


def _flag_mask(lay):
    lo = hi = 0
    for b in list(lay["flag_bit"]) + list(lay["hot_bit"]):
        if b >= 0:
            if b < 64:
                lo |= 1 << b
            else:
                hi |= 1 << (b - 64)
    return np.uint64(lo), np.uint64(hi)


def check_format(dims, idx, vals, at):
    ex = at.export()
    lay = at.layout()
    st = at.stats()
    L = st["nparts"]
    o = oracle_format(dims, idx, vals, L)
    kw = lay["key_words"]
    flo, fhi = _flag_mask(lay)
    keys = ex["keys"].copy()
    keys[:, 0] &= ~flo
    if kw == 2:
        keys[:, 1] &= ~fhi
    else:
        assert (o["keys"][:, 1] == 0).all()
    assert (keys == o["keys"][:, :kw]).all(), "keys differ"
    assert (ex["perm"].astype(np.int64) == o["perm"]).all(), "permutation differs"
    assert (ex["vals"] == o["vals"]).all(), "values differ"
    assert (ex["bounds"] == o["bounds"]).all(), "bounds differ"
    assert (ex["intervals"].astype(np.uint64) == o["intervals"]).all(), "intervals differ"
    for n in range(len(dims)):
        assert st["distinct"][n] == len(np.unique(idx[n])) if len(vals) else st["distinct"][n] == 0
        b = lay["flag_bit"][n]
        if b >= 0:
            word = ex["keys"][:, b // 64]
            got = (word >> np.uint64(b % 64)) & np.uint64(1)
            ref = oracle.flags(o["coords"], dims[n], n, o["bounds"])
            assert (got.astype(np.uint8) == ref).all(), "flags differ in mode %d" % n
        check_hot(at, n, o["coords"][:, n].astype(np.int64), lay, ex["keys"], dims[n])
    return ex, o


def expected_hot_rows(rows_in_alto_order, I):
    """The hot-row rule: count every 16th nonzero in ALTO order per row; keep
    the rows whose count reaches the smallest power of two 2^b (b >= 1) that
    leaves at most 1024 rows; hottest first, ties by row."""
    c = np.bincount(rows_in_alto_order[::16], minlength=I)
    nz = c[c > 0]
    if nz.size == 0:
        return np.zeros(0, np.int64)
    lg = np.floor(np.log2(nz)).astype(np.int64)
    hist = np.bincount(lg, minlength=33)
    b = 1
    above = hist[1:].sum()
    while b < 33 and above > 1024:
        above -= hist[b]
        b += 1
    if b >= 33 or above == 0:
        return np.zeros(0, np.int64)
    rows = np.flatnonzero(c >= (1 << b))
    order = np.lexsort((rows, -c[rows]))
    return rows[order]


def check_hot(at, n, rows_sorted, lay, keys, I):
    hot = at.hot_rows(n).astype(np.int64)
    assert (hot == expected_hot_rows(rows_sorted, I)).all(), "hot rows differ in mode %d" % n
    b = lay["hot_bit"][n]
    if b >= 0:
        got = (keys[:, b // 64] >> np.uint64(b % 64)) & np.uint64(1)
        ref = np.isin(rows_sorted, hot) if hot.size else np.zeros(len(rows_sorted), bool)
        assert (got.astype(bool) == ref).all(), "hot flags differ in mode %d" % n


@pytest.mark.parametrize("name,nnz", [("uniform3d-64x128x256", None), ("zipf3d-4Mx4Mx30k", 300_000),
                                      ("clustered4d-12kx60kx5Mx100", 300_000), ("long5d-2^20x3-2^16x2", 200_000)])
def test_format_configs(name, nnz):
    cfg = synth.scaled(name, nnz=nnz) if nnz else synth.CONFIGS[name]
    dims, idx, vals = synth.tensor(cfg)
    at = make(dims, idx, vals)
    check_format(dims, idx, vals, at)
    if name.startswith("long5d"):
        assert at.layout()["key_words"] == 2


def test_forced_128bit_keys():
    dims, idx, vals = synth.tensor(synth.CONFIGS["uniform3d-64x128x256"])
    at = make(dims, idx, vals, key_bits=128)
    assert at.layout()["key_words"] == 2
    check_format(dims, idx, vals, at)


@pytest.mark.parametrize("M", [0, 1, 2, 31, 33, 4095, 4097, 12_345])
def test_ragged_sizes(M):
    rng = np.random.default_rng(M)
    dims = (300, 17, 1000)
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.random(M).astype(np.float32)
    at = make(dims, idx, vals)
    check_format(dims, idx, vals, at)


def test_duplicates_keep_input_order():
    rng = np.random.default_rng(5)
    dims = (8, 9, 10)
    M = 20_000                      # 720 cells: every cell repeats
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.random(M).astype(np.float64)
    at = make(dims, idx, vals)
    ex, o = check_format(dims, idx, vals, at)
    k = ex["keys"][:, 0]
    ties = k[1:] == k[:-1]
    assert ties.any() and (ex["perm"][1:][ties] > ex["perm"][:-1][ties]).all()


@pytest.mark.parametrize("dims", [(5,), (1, 1, 1), (3, 1, 7), (2, 3, 4, 5, 6, 7, 8, 9), (2 ** 32, 3)])
def test_orders_and_extreme_lengths(dims):
    rng = np.random.default_rng(len(dims))
    M = 3000
    idx = [rng.integers(0, d, M, dtype=np.int64).astype(np.uint32) for d in dims]
    idx[0][0] = np.uint32(dims[0] - 1)
    vals = rng.random(M).astype(np.float32)
    at = make(dims, idx, vals)
    check_format(dims, idx, vals, at)


def test_flags_for_low_reuse_modes():
    rng = np.random.default_rng(7)
    dims = (20, 50_000, 40_000)     # reuse 1000, 0.4, 0.5 -> modes 1, 2 flagged
    M = 20_000
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.random(M).astype(np.float32)
    at = make(dims, idx, vals, nparts=37)
    lay = at.layout()
    assert lay["flag_bit"][0] == -1 and lay["flag_bit"][1] >= 0 and lay["flag_bit"][2] >= 0
    check_format(dims, idx, vals, at)


def test_nparts_override_and_int64_host_inputs():
    dims, idx, vals = synth.tensor(synth.scaled("zipf3d-4Mx4Mx30k", nnz=50_000))
    from paper_2102_10245_gb300 import AltoTensor
    # int64 indices, pinned host memory
    hidx = [torch.from_numpy(a.astype(np.int64)).pin_memory() for a in idx]
    at = AltoTensor(dims, hidx, torch.from_numpy(vals).pin_memory(), nparts=13)
    assert at.stats()["nparts"] == 13
    check_format(dims, idx, vals, at)
    # pageable host memory
    at2 = AltoTensor(dims, [torch.from_numpy(a.astype(np.int64)) for a in idx], torch.from_numpy(vals), nparts=7)
    check_format(dims, idx, vals, at2)


def test_max_interval_and_reuse_stats():
    dims, idx, vals = synth.tensor(synth.CONFIGS["uniform3d-64x128x256"])
    at = make(dims, idx, vals)
    st = at.stats()
    ex = at.export()
    widths = ex["intervals"][:, :, 1].astype(np.int64) - ex["intervals"][:, :, 0] + 1
    assert st["max_interval"] == list(widths.max(0))
    assert st["reuse"] == [len(vals) / d for d in dims]
