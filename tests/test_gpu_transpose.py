"""Sparse tensor transposition on the GPU (Sec. 5) against the oracle.

The ALTO positions, input positions, coordinates (in the new mode order) and
values of the result are compared bit-exact with ``oracle.transpose``: full
mode permutations, one- and two-mode partial orders (ties in ALTO order),
32-, 64-, 96- and 128-bit stored keys, sort keys of one and two words with a
coordinate straddling the word boundary, duplicates, orders 1 and 8, a
length-1 mode, a 2^32-long mode and the empty tensor.  At 150M nonzeros the
result is checked through properties that fix it uniquely.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import dev, dev_idx, make

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32).astype(np.int64)


def check(dims, idx, vals, at, modes, idx_dtype=torch.int64):
    got = at.transpose(modes, order=True, idx_dtype=idx_dtype)
    torch.cuda.synchronize()
    order, src = oracle.transpose(dims, idx, modes)
    assert np.array_equal(_u32(got["order"]), order), ("order", modes)
    assert np.array_equal(_u32(got["src"]), src), ("src", modes)
    omodes = list(modes) + [m for m in range(len(dims)) if m not in modes]
    for j, m in enumerate(omodes):
        g = got["idx"][j].cpu().numpy()
        g = g.view(np.uint32).astype(np.int64) if idx_dtype == torch.int32 else g
        assert np.array_equal(g, np.asarray(idx[m], np.int64)[src]), ("idx", modes, j)
    v = got["vals"]
    ref = np.asarray(vals)[src]
    if v.dtype == torch.bfloat16:
        assert np.array_equal(v.to(torch.float64).cpu().numpy(), ref.astype(np.float64))
    else:
        assert np.array_equal(v.cpu().numpy(), ref), ("vals", modes)


def _sels(N):
    s = [list(p) for p in itertools.permutations(range(N))][:6]
    s += [[m] for m in range(N)]
    if N > 2:
        s += [[N - 1, 0], [1, N - 1]]
    return s


def test_uniform_small_every_selection(alto_lib):
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    at = make(dims, idx, vals)
    assert at.key_bytes() == 4
    for modes in _sels(3):
        check(dims, idx, vals, at, modes)
    check(dims, idx, vals, at, [2, 1, 0], idx_dtype=torch.int32)
    at.close()


@pytest.mark.parametrize("name,nnz,kb", [("zipf3d-4Mx4Mx30k", 200_000, 8),
                                          ("clustered4d-12kx60kx5Mx100", 150_000, 8),
                                          ("long5d-2^20x3-2^16x2", 100_000, 12)])
def test_scaled_configs(alto_lib, name, nnz, kb):
    cfg = synth.scaled(name, nnz=nnz)
    dims, idx, vals = synth.tensor(cfg)
    at = make(dims, idx, vals)
    assert at.key_bytes() == kb
    N = len(dims)
    sels = [list(range(N))[::-1], [N - 1], [0], [1, N - 1]]
    if N == 5:
        # b = 20,20,20,16,16: mode 3 sits at bits 60..75 of the 92-bit sort key
        sels.append([4, 3, 2, 1, 0])
    for modes in sels:
        check(dims, idx, vals, at, modes)
    at.close()


def test_bf16_values_and_forced_128bit_keys(alto_lib):
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=50_000)
    dims, idx, vals = synth.tensor(cfg)
    from paper_2102_10245_gb300 import AltoTensor
    v16 = torch.from_numpy(np.asarray(vals, np.float32)).to(torch.bfloat16)
    at = AltoTensor(dims, dev_idx(idx), v16.cuda())
    ref = v16.to(torch.float64).numpy()
    for modes in ([2, 0, 1], [1]):
        check(dims, idx, ref, at, modes)
    at.close()
    at = make(dims, idx, vals, key_bits=128)
    assert at.key_bytes() == 16
    check(dims, idx, vals, at, [2, 1, 0])
    at.close()


def test_duplicates_keep_input_order(alto_lib):
    rng = np.random.default_rng(21)
    dims = (5, 6, 7)
    M = 5000
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.random(M)
    at = make(dims, idx, vals)
    for modes in ([0, 1, 2], [2, 1, 0], [2], [1, 0]):
        check(dims, idx, vals, at, modes)
    at.close()


@pytest.mark.parametrize("dims,M", [((1000,), 700), ((3,) * 8, 2000), ((1, 50, 60), 1500), ((2 ** 32, 5), 3000),
                                    ((4, 8, 2), 1)])
def test_edge_shapes(alto_lib, dims, M):
    rng = np.random.default_rng(len(dims) + M)
    idx = [rng.integers(0, d, M, dtype=np.uint64).astype(np.uint32) for d in dims]
    vals = rng.random(M)
    at = make(dims, idx, vals)
    N = len(dims)
    for modes in ([list(range(N))[::-1], [0]] + ([[N - 1, 0]] if N > 1 else [])):
        check(dims, idx, vals, at, modes)
    at.close()


def test_empty_tensor_and_argument_errors(alto_lib):
    from paper_2102_10245_gb300 import AltoError
    dims = (4, 5, 6)
    idx = [np.zeros(0, np.uint32) for _ in dims]
    at = make(dims, idx, np.zeros(0))
    got = at.transpose([2, 0, 1], order=True)
    assert got["src"].numel() == 0 and all(a.numel() == 0 for a in got["idx"])
    at.close()
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    at = make(dims, idx, vals)
    for bad in ([], [0, 0], [3], [-1], [0, 1, 2, 0]):
        with pytest.raises(AltoError):
            at.transpose(bad)
    at.close()


@pytest.mark.slow
def test_full_size_zipf_properties(alto_lib):
    """150M distinct nonzeros: the result of the full transposition is a
    permutation whose coordinates are the input's at those positions and
    strictly increase in the new lexicographic order -- which fixes it
    uniquely; the one-mode partial order is non-decreasing in that mode with
    ties in ascending ALTO position."""
    cfg = synth.CONFIGS["zipf3d-4Mx4Mx30k"]
    d = torch.device("cuda", 0)
    dims, idx_d, vals_d = synth.tensor_torch(cfg, d)
    from paper_2102_10245_gb300 import AltoTensor
    at = AltoTensor(dims, idx_d, vals_d)
    M = vals_d.numel()
    modes = [2, 0, 1]
    got = at.transpose(modes)
    src = got["src"].to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(torch.bincount(src, minlength=M), torch.ones(M, dtype=torch.int64, device=d))
    for j, m in enumerate(modes):
        inp = idx_d[m].to(torch.int64) & 0xFFFFFFFF
        assert torch.equal(got["idx"][j], inp[src])
    assert torch.equal(got["vals"], vals_d[src])
    lin = (got["idx"][0] * dims[0] + got["idx"][1]) * dims[1] + got["idx"][2]
    assert bool((lin[1:] > lin[:-1]).all())
    del got, lin, src
    part = at.transpose([0], order=True, src=False, vals=False)
    i0, o = part["idx"][0], part["order"].to(torch.int64) & 0xFFFFFFFF
    assert bool((i0[1:] >= i0[:-1]).all())
    tie = i0[1:] == i0[:-1]
    assert bool((o[1:][tie] > o[:-1][tie]).all())
    assert torch.equal(torch.bincount(o, minlength=M), torch.ones(M, dtype=torch.int64, device=d))
    at.close()
