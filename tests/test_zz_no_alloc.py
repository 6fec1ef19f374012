"""The allocation-free linearization entry point (alto_linearize_noalloc).

Callers that cannot allocate device memory -- code running under CUDA-graph
stream capture, services that reserve all device memory up front, embedders
whose allocator belongs to another runtime -- use this entry point.  It must
produce exactly the keys and permutation that alto_create computes, call
after call, although every call reuses the same fixed scratch array.  The
file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _noalloc(dims, idx_dev, kw):
    from paper_2102_10245_gb300 import alto
    M = idx_dev[0].shape[0]
    keys = torch.empty((M, kw), dtype=torch.int64, device="cuda")
    perm = torch.empty(M, dtype=torch.int32, device="cuda")
    ptrs = (ctypes.c_void_p * len(dims))(*[a.data_ptr() for a in idx_dev])
    d = (ctypes.c_uint64 * len(dims))(*dims)
    st = alto.lib().alto_linearize_noalloc(len(dims), d, M, ptrs, 4, ctypes.c_void_p(keys.data_ptr()),
                                           ctypes.c_void_p(perm.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32)


def _reference(dims, idx, vals):
    from paper_2102_10245_gb300 import AltoTensor
    at = AltoTensor(dims, [torch.from_numpy(a.view(np.int32)).cuda() for a in idx],
                    torch.from_numpy(vals).cuda(), use_flags=False)
    ex = at.export()
    return ex["keys"], ex["perm"], at.layout()["key_words"]


@pytest.mark.parametrize("name,nnz", [("zipf3d-4Mx4Mx30k", 200_000), ("long5d-2^20x3-2^16x2", 150_000)])
def test_noalloc_matches_create_on_two_calls(name, nnz):
    from paper_2102_10245_gb300 import alto
    cfgs = [synth.scaled(name, nnz=nnz), synth.scaled(name, nnz=nnz // 3, seed=77)]
    for cfg in cfgs:     # two calls in a row, the second smaller than the first
        dims, idx, vals = synth.tensor(cfg)
        rk, rp, kw = _reference(dims, idx, vals)
        st, k, p = _noalloc(dims, [torch.from_numpy(a.view(np.int32)).cuda() for a in idx], kw)
        assert st == alto.ALTO_OK, alto.lib().alto_last_error()
        assert (k == rk).all() and (p == rp).all()


def test_noalloc_rejects_more_than_the_fixed_limit():
    from paper_2102_10245_gb300 import alto
    M = 262_144 + 1
    idx = [torch.zeros(M, dtype=torch.int32, device="cuda") for _ in range(3)]
    st, _, _ = _noalloc((4, 4, 4), idx, 1)
    assert st == alto.ALTO_EINVAL
