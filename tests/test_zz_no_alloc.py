"""The allocation-free linearization entry point (alto_linearize_noalloc).

Callers that cannot allocate device memory -- services that reserve all
device memory up front, embedders whose allocator belongs to another runtime
-- use this entry point.  Its keys and permutation must be the ALTO keys and
the stable order that the oracle computes from the paper's definition (Sec.
3.1), and those alto_create gives for the same input, call after call, although
every call reuses the same fixed scratch array, and a call must not allocate
device memory.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import make

pytestmark = pytest.mark.gpu


def _kw(dims):
    from paper_2102_10245_gb300 import alto
    return alto.layout_for_dims(dims)[2]


def _noalloc(dims, idx_dev, keys, perm):
    from paper_2102_10245_gb300 import alto
    M = idx_dev[0].shape[0]
    ptrs = (ctypes.c_void_p * len(dims))(*[a.data_ptr() for a in idx_dev])
    d = (ctypes.c_uint64 * len(dims))(*dims)
    return alto.lib().alto_linearize_noalloc(len(dims), d, M, ptrs, 4, ctypes.c_void_p(keys.data_ptr()),
                                             ctypes.c_void_p(perm.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("name,nnz", [("zipf3d-4Mx4Mx30k", 200_000), ("long5d-2^20x3-2^16x2", 150_000)])
def test_noalloc_matches_oracle_on_two_calls(name, nnz):
    from paper_2102_10245_gb300 import alto
    cfgs = [synth.scaled(name, nnz=nnz), synth.scaled(name, nnz=nnz // 3, seed=77)]
    # a first call loads the library's kernels and its fixed array on this
    # device (module loading, not an allocation by the call): it is not measured
    dims, idx, _ = synth.tensor(cfgs[1])
    M = len(idx[0])
    assert _noalloc(dims, [torch.from_numpy(a.view(np.int32)).cuda() for a in idx],
                    torch.empty((M, _kw(dims)), dtype=torch.int64, device="cuda"),
                    torch.empty(M, dtype=torch.int32, device="cuda")) == alto.ALTO_OK
    for cfg in cfgs:     # two calls in a row, the second smaller than the first
        dims, idx, vals = synth.tensor(cfg)
        ref_keys = oracle.encode(dims, idx)
        ref_perm = oracle.sort_perm(ref_keys)
        kw = _kw(dims)
        M = len(vals)
        keys = torch.empty((M, kw), dtype=torch.int64, device="cuda")
        perm = torch.empty(M, dtype=torch.int32, device="cuda")
        idx_dev = [torch.from_numpy(a.view(np.int32)).cuda() for a in idx]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _noalloc(dims, idx_dev, keys, perm)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == alto.ALTO_OK, alto.lib().alto_last_error()
        assert free1 == free0, "the call allocated device memory (%d bytes)" % (free0 - free1)
        k = keys.cpu().numpy().view(np.uint64).reshape(M, kw)
        p = perm.cpu().numpy().view(np.uint32)
        assert (p == ref_perm).all()
        assert (k == ref_keys[ref_perm][:, :kw]).all()
        # the existing entry point on the same input gives the same result:
        # alto_create's keys (its helper-flag bits masked off) and permutation
        at = make(dims, idx, vals)
        ex, lay = at.export(), at.layout()
        at.close()
        ck = ex["keys"].copy()
        for b in list(lay["flag_bit"]) + list(lay["hot_bit"]):
            if b >= 0:
                ck[:, b // 64] &= ~np.uint64(1 << (b % 64))
        assert (p == ex["perm"]).all()
        assert (k == ck).all()


def test_noalloc_rejects_more_than_the_fixed_limit():
    from paper_2102_10245_gb300 import alto
    M = 262_144 + 1
    idx = [torch.zeros(M, dtype=torch.int32, device="cuda") for _ in range(3)]
    keys = torch.empty((1, 1), dtype=torch.int64, device="cuda")
    perm = torch.empty(1, dtype=torch.int32, device="cuda")
    assert _noalloc((4, 4, 4), idx, keys, perm) == alto.ALTO_EINVAL
