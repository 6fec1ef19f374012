"""Gram matrices U^T U (Sec. 2.2: the factors of CP-ALS's system matrix V) on
the tensor cores (tcgen05, BF16 factors) and on the CUDA cores, against the
plain FP64 product of the same (BF16-rounded) values.

Bound: BF16 x BF16 products are exact in FP32; an FP32 sum runs over at most
k of them (any order, rounding to nearest or toward zero) and the partial
sums are added in FP64.  So |G - G_ref| <= (k 2^-23 + I 2^-52) (|U|^T |U|)
entrywise: k = 1024 on the tensor cores (the accumulator is moved into FP64
every 1024 rows), k = I on the CUDA cores.  A layout or descriptor mistake
gives O(1) errors.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _bf16_factor(I, R, seed):
    g = torch.Generator().manual_seed(seed)
    u = torch.randn(I, R, generator=g, dtype=torch.float32).to(torch.bfloat16)
    return u.cuda(), u.to(torch.float64).numpy()


def _check(G, U64, k):
    G = G.cpu().numpy()
    ref = U64.T @ U64
    I = U64.shape[0]
    bound = (k * 2.0 ** -23 + I * 2.0 ** -52) * (np.abs(U64).T @ np.abs(U64)) + 1e-300
    assert np.all(np.abs(G - ref) <= bound), float(np.max(np.abs(G - ref) / bound))
    return float(np.linalg.norm(G - ref) / max(np.linalg.norm(ref), 1e-300))


@pytest.mark.parametrize("R", [8, 16, 32, 64])
@pytest.mark.parametrize("I", [1, 63, 64, 65, 1000, 100_003])
def test_tensor_core_gram_matches_fp64(alto_lib, R, I):
    from paper_2102_10245_gb300 import gram, GRAM_TENSOR_CORES, GRAM_CUDA_CORES
    U, U64 = _bf16_factor(I, R, 1000 * R + I)
    e_tc = _check(gram(U, GRAM_TENSOR_CORES), U64, min(I, 1024))
    e_cc = _check(gram(U, GRAM_CUDA_CORES), U64, I)
    assert e_tc < 1e-5 and e_cc < 1e-5


def test_tensor_core_gram_long_factor(alto_lib):
    """4M rows (the long modes of the 4M x 4M x 30k tensor) at R = 32."""
    from paper_2102_10245_gb300 import gram, GRAM_TENSOR_CORES
    U, U64 = _bf16_factor(4_000_000, 32, 7)
    e = _check(gram(U, GRAM_TENSOR_CORES), U64, 1024)
    print("tensor-core Gram, 4M x 32: relative error %.2e" % e)
    assert e < 1e-5


def test_gram_edge_cases_and_errors(alto_lib):
    from paper_2102_10245_gb300 import gram, AltoError, GRAM_AUTO, GRAM_TENSOR_CORES
    U = torch.zeros(0, 32, dtype=torch.bfloat16, device="cuda")
    assert torch.equal(gram(U, GRAM_TENSOR_CORES), torch.zeros(32, 32, dtype=torch.float64, device="cuda"))
    with pytest.raises(AltoError):
        gram(torch.zeros(10, 32, dtype=torch.float32, device="cuda"), GRAM_TENSOR_CORES)
    with pytest.raises(AltoError):
        gram(torch.zeros(10, 24, dtype=torch.bfloat16, device="cuda"), GRAM_TENSOR_CORES)
    # automatic engine: any R and dtype
    for dt in (torch.float32, torch.float64, torch.bfloat16):
        U = torch.randn(500, 24, device="cuda").to(dt)
        U64 = U.to(torch.float64).cpu().numpy()
        _check(gram(U, GRAM_AUTO), U64, 500)


def test_cpals_bf16_engines_agree(alto_lib):
    """CP-ALS with BF16 factors: tensor-core and CUDA-core Grams give the
    same fits to BF16 accuracy."""
    import synth
    from helpers import make
    from paper_2102_10245_gb300 import GRAM_CUDA_CORES, GRAM_TENSOR_CORES
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=300_000)
    cfg["dims"] = (200_000, 200_000, 3000)
    dims, idx, vals = synth.tensor(cfg)
    at = make(dims, idx, vals.astype(np.float32))
    fits = {}
    for eng in (GRAM_CUDA_CORES, GRAM_TENSOR_CORES):
        at.set_gram_engine(eng)
        U = [u.to(torch.bfloat16) for u in synth.factors_torch(dict(cfg, rank=32), "cuda", torch.float32)]
        _, f = at.cpals(U, 4)
        fits[eng] = f
    assert np.allclose(fits[GRAM_CUDA_CORES], fits[GRAM_TENSOR_CORES], rtol=1e-2, atol=1e-3), fits
    at.close()
