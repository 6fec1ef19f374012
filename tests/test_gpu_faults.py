"""Failure paths of the boundary, all made on the host or with inputs the
kernels check: an index outside its mode (the encoder records ALTO_ERANGE
and substitutes 0, so nothing reads out of bounds), a device allocator that
fails (ALTO_ENOMEM through the allocation hook, everything already allocated
handed back), invalid orders and lengths, mismatched dtypes, and a handle
that stays usable after each error.  None of these faults or traps the GPU."""
import numpy as np
import pytest
import torch

from helpers import dev, dev_idx, make

pytestmark = pytest.mark.gpu


def _small(seed=0, dims=(10, 20, 30), M=500):
    rng = np.random.default_rng(seed)
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.random(M).astype(np.float32)
    return dims, idx, vals


def test_index_out_of_range_reports_erange(alto_lib):
    from paper_2102_10245_gb300 import AltoError
    dims, idx, vals = _small()
    idx[1][17] = np.uint32(dims[1])          # one past the end of mode 1
    with pytest.raises(AltoError) as e:
        make(dims, idx, vals)
    assert e.value.status == 7               # ALTO_ERANGE
    # the context and the library stay usable
    idx[1][17] = np.uint32(0)
    at = make(dims, idx, vals)
    assert at.stats()["nnz"] == len(vals)


def test_failing_allocator_reports_enomem_and_returns_memory(alto_lib):
    from paper_2102_10245_gb300 import AltoError, AltoTensor
    dims, idx, vals = _small(1)
    live = {}
    calls = {"n": 0}

    def alloc(nbytes, ctx):
        calls["n"] += 1
        if calls["n"] > 3:                   # the fourth request fails
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes))
        live[p] = nbytes
        return p

    def free(ptr, ctx):
        if ptr:
            live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

    with pytest.raises(AltoError) as e:
        AltoTensor(dims, dev_idx(idx), dev(vals), allocator=(alloc, free))
    assert e.value.status == 2               # ALTO_ENOMEM
    assert calls["n"] == 4 and not live      # every successful allocation was returned
    at = AltoTensor(dims, dev_idx(idx), dev(vals))
    assert at.stats()["nnz"] == len(vals)


@pytest.mark.parametrize("dims", [(5,) * 9, (10, 0, 30)])
def test_bad_order_or_length_reports_einval(alto_lib, dims):
    from paper_2102_10245_gb300 import AltoError
    M = 100
    idx = [np.zeros(M, np.uint32) for _ in dims]
    vals = np.ones(M, np.float32)
    with pytest.raises(AltoError) as e:
        make(dims, idx, vals)
    assert e.value.status == 1               # ALTO_EINVAL


def test_mismatched_dtypes_report_einval(alto_lib):
    from paper_2102_10245_gb300 import AltoError, Batch
    dims, idx, vals = _small(2)
    at = make(dims, idx, vals)               # FP32 values
    R = 8
    U64 = [torch.zeros(d, R, dtype=torch.float64, device="cuda") for d in dims]
    with pytest.raises(AltoError) as e:      # FP64 factors need FP64 values
        at.mttkrp(0, U64)
    assert e.value.status == 1
    out = torch.empty(dims[0], R, dtype=torch.float64, device="cuda")
    with pytest.raises(AltoError) as e:
        Batch([(at, 0, U64, out)])
    assert e.value.status == 1
    # the handle still computes
    U = [torch.ones(d, R, device="cuda") for d in dims]
    got = at.mttkrp(0, U)
    torch.cuda.synchronize()
    ref = np.zeros((dims[0], R))
    np.add.at(ref, idx[0].astype(np.int64), vals.astype(np.float64)[:, None])
    assert np.allclose(got.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)
