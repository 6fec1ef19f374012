"""Shared helpers of the GPU parity tests: moving seeded inputs to the
device, running the oracle on the same inputs, and error measures."""
import numpy as np
import torch

import oracle


def rel_err(got, ref):
    """Relative Frobenius error ||got - ref|| / ||ref|| (absolute if ref = 0)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(got - ref)
    n = np.linalg.norm(ref)
    return d / n if n > 0 else d


def dev_idx(idx, dtype=torch.int32):
    """uint32 numpy index arrays -> CUDA tensors holding the same bits."""
    out = []
    for a in idx:
        a = np.ascontiguousarray(a)
        if dtype == torch.int32:
            out.append(torch.from_numpy(a.astype(np.uint32).view(np.int32)).cuda())
        else:
            out.append(torch.from_numpy(a.astype(np.int64)).cuda())
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(dims, idx, vals, **kw):
    from paper_2102_10245_gb300 import AltoTensor
    return AltoTensor(dims, dev_idx(idx), dev(vals), **kw)


def oracle_format(dims, idx, vals, L):
    """Keys, permutation, values, bounds, intervals and decoded coordinates
    of the ALTO tensor, all from the oracle."""
    keys = oracle.encode(dims, idx)
    perm = oracle.sort_perm(keys)
    ks = keys[perm]
    coords = oracle.decode(dims, ks)
    bounds = oracle.partition(len(perm), L)
    ivl = oracle.intervals(coords, bounds)
    return dict(keys=ks, perm=perm, vals=np.asarray(vals)[perm], bounds=bounds, intervals=ivl, coords=coords)


def factors_np(dims, R, seed, dtype=np.float32, dist="normal"):
    rng = np.random.default_rng(seed)
    if dist == "normal":
        return [rng.standard_normal((d, R)).astype(dtype) for d in dims]
    return [rng.random((d, R)).astype(dtype) for d in dims]


def to_bf16_exact(f):
    """BF16-rounded copy of an FP32 array (as torch bf16 on the GPU) and the
    exact FP64 value of the rounded entries (for the oracle)."""
    t = torch.from_numpy(np.ascontiguousarray(f)).to(torch.bfloat16)
    return t.cuda(), t.to(torch.float64).numpy()
