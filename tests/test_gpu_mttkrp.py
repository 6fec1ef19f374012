"""MTTKRP over the ALTO format on the GPU against the FP64 oracle (Sec. 2.2,
Alg. 1-2): every accumulation variant, FP64 / FP32 / BF16-factor paths,
orders 1-8, specialised and generic ranks.  Tolerances (relative Frobenius
error): 1e-12 for FP64, 1e-5 for FP32, 1e-2 for BF16 factors against the
unrounded factors (and 1e-5 against the BF16-rounded ones, which isolates the
FP32 accumulation)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import dev, factors_np, make, rel_err, to_bf16_exact

pytestmark = pytest.mark.gpu

VARIANTS = [1, 2, 3, 4]   # atomic, warpagg, smem, temp
TOL = {np.float64: 1e-12, np.float32: 1e-5}


def run_all_modes(at, dims, idx, vals, U, variant, tol, label):
    Ud = [dev(u) for u in U]
    for n in range(len(dims)):
        at.set_variant(n, variant)
        fs = Ud if len(dims) == 1 else [u if m != n else None for m, u in enumerate(Ud)]
        got = at.mttkrp(n, fs)
        torch.cuda.synchronize()
        ref = oracle.mttkrp(dims, idx, vals, U, n)
        err = rel_err(got.cpu().numpy(), ref)
        print("%s mode %d variant %d: rel err %.3e" % (label, n, variant, err))
        assert err <= tol, (label, n, variant, err)


@pytest.mark.parametrize("variant", VARIANTS)
def test_small_uniform_fp64(variant):
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    at = make(dims, idx, vals)
    run_all_modes(at, dims, idx, vals, U, variant, 1e-12, "uniform3d fp64")


@pytest.mark.parametrize("name,nnz", [("zipf3d-4Mx4Mx30k", 400_000), ("clustered4d-12kx60kx5Mx100", 400_000),
                                      ("long5d-2^20x3-2^16x2", 300_000)])
@pytest.mark.parametrize("variant", VARIANTS)
def test_scaled_configs_fp32(name, nnz, variant):
    cfg = synth.scaled(name, nnz=nnz)
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    at = make(dims, idx, vals)
    run_all_modes(at, dims, idx, vals, U, variant, 1e-5, name + " fp32")


@pytest.mark.parametrize("variant", VARIANTS)
def test_bf16_factors(variant):
    cfg = synth.scaled("clustered4d-12kx60kx5Mx100", nnz=300_000)
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    at = make(dims, idx, vals)
    pairs = [to_bf16_exact(u) for u in U]
    Ub = [p[0] for p in pairs]
    Ur = [p[1] for p in pairs]
    for n in range(len(dims)):
        at.set_variant(n, variant)
        got = at.mttkrp(n, Ub).cpu().numpy()
        e_round = rel_err(got, oracle.mttkrp(dims, idx, vals, Ur, n))
        e_full = rel_err(got, oracle.mttkrp(dims, idx, vals, U, n))
        print("bf16 mode %d variant %d: err vs rounded %.3e, vs fp32 factors %.3e" % (n, variant, e_round, e_full))
        assert e_round <= 1e-5 and e_full <= 1e-2


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("R", [1, 3, 8, 16, 32, 64, 100])
def test_orders_and_ranks(N, R):
    rng = np.random.default_rng(100 * N + R)
    dims = tuple(int(x) for x in rng.integers(2, 60, N))
    M = 5000
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.standard_normal(M).astype(np.float32)
    U = factors_np(dims, R, seed=R)
    at = make(dims, idx, vals)
    for v in (1, 2, 3, 4):
        run_all_modes(at, dims, idx, vals, U, v, 1e-5, "N=%d R=%d" % (N, R))


def test_fp64_generic_rank_and_order():
    rng = np.random.default_rng(3)
    dims = (7, 11, 5, 9, 4, 6)
    M = 4000
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.standard_normal(M)
    U = factors_np(dims, 24, seed=1, dtype=np.float64)
    at = make(dims, idx, vals)
    run_all_modes(at, dims, idx, vals, U, 0, 1e-12, "fp64 N=6 R=24")


def test_duplicates_are_summed():
    rng = np.random.default_rng(4)
    dims = (6, 7, 8)
    M = 3000
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.standard_normal(M)
    U = factors_np(dims, 16, seed=2, dtype=np.float64)
    at = make(dims, idx, vals)
    for v in VARIANTS:
        run_all_modes(at, dims, idx, vals, U, v, 1e-12, "duplicates")


def test_output_is_overwritten_and_empty_tensor():
    dims = (10, 20, 30)
    idx = [np.zeros(0, np.uint32)] * 3
    vals = np.zeros(0, np.float32)
    at = make(dims, idx, vals)
    U = [dev(f) for f in factors_np(dims, 8, seed=0)]
    out = torch.full((10, 8), 7.0, device="cuda")
    at.mttkrp(0, U, out=out)
    assert (out == 0).all()
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    Uf = synth.factors(cfg)
    at = make(dims, idx, vals)
    out = torch.full((256, 16), 3.0, device="cuda", dtype=torch.float64)
    at.mttkrp(2, [dev(u) for u in Uf], out=out)
    assert rel_err(out.cpu().numpy(), oracle.mttkrp(dims, idx, vals, Uf, 2)) <= 1e-12


def test_dtype_mismatch_rejected():
    from paper_2102_10245_gb300 import AltoError
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    at = make(dims, idx, vals)            # FP64 values
    U = [dev(f) for f in factors_np(dims, 8, seed=0)]   # FP32 factors
    with pytest.raises(AltoError) as e:
        at.mttkrp(0, U)
    assert e.value.status == 1
    with pytest.raises(AltoError):
        at.set_variant(5, 1)


def _bf16_values(vals):
    """BF16-rounded copy of FP32 values (torch bf16 on the GPU) and their
    exact FP64 values."""
    t = torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda(), t.to(torch.float64).numpy()


@pytest.mark.parametrize("variant", VARIANTS + [5])
@pytest.mark.parametrize("fdt", ["f32", "bf16"])
def test_bf16_values(variant, fdt):
    """Values stored as BF16 (2-byte value stream), FP32 accumulation: within
    1e-5 of the oracle on the BF16-rounded values (and rounded factors), 1e-2
    of the oracle on the FP32 values; the exported values are the rounded
    ones in ALTO order."""
    from paper_2102_10245_gb300 import AltoTensor
    from helpers import dev_idx
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=300_000)
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    vb, vr = _bf16_values(vals)
    at = AltoTensor(dims, dev_idx(idx), vb)
    if fdt == "bf16":
        pairs = [to_bf16_exact(u) for u in U]
        Ud, Ur = [p[0] for p in pairs], [p[1] for p in pairs]
    else:
        Ud, Ur = [dev(u) for u in U], [u.astype(np.float64) for u in U]
    ex = at.export()
    assert np.array_equal(ex["vals"].astype(np.float64), vr[ex["perm"]])
    for n in range(len(dims)):
        at.set_variant(n, variant)
        got = at.mttkrp(n, Ud).cpu().numpy()
        e_round = rel_err(got, oracle.mttkrp(dims, idx, vr, Ur, n))
        e_full = rel_err(got, oracle.mttkrp(dims, idx, vals, U, n))
        print("bf16 values, %s factors, mode %d variant %d: %.3e vs rounded, %.3e vs fp32" % (fdt, n, variant,
                                                                                             e_round, e_full))
        assert e_round <= 1e-5 and e_full <= 1e-2


@pytest.mark.parametrize("variant", [1, 2])
def test_segment_count_override(variant):
    """alto_set_parts: any segment count (coarser, finer, one segment, more
    than nnz) gives the same MTTKRP for ATOMIC and WARPAGG; 0 restores L."""
    cfg = synth.scaled("clustered4d-12kx60kx5Mx100", nnz=200_000)
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    at = make(dims, idx, vals)
    Ud = [dev(u) for u in U]
    L = at.stats()["nparts"]
    for parts in (max(1, L // 4), L * 4, 1, 10 * len(vals), 0):
        for n in range(len(dims)):
            at.set_variant(n, variant)
            at.set_parts(n, parts)
            got = at.mttkrp(n, Ud).cpu().numpy()
            err = rel_err(got, oracle.mttkrp(dims, idx, vals, U, n))
            assert err <= 1e-5, (parts, n, err)


def test_generic_variant_forced():
    """ALTO_VAR_GENERIC runs the runtime-rank kernel on a specialised shape."""
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=100_000)
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    at = make(dims, idx, vals)
    run_all_modes(at, dims, idx, vals, U, 5, 1e-5, "generic forced")
    assert at.resolve_variant(0, 32, 1, 5) == 5
