"""CP-ALS over ALTO MTTKRP on the GPU against the oracle's Kolda-Bader
CP-ALS (Sec. 2.2): per-iteration fit, lambda and factors."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import dev, make, rel_err, to_bf16_exact

pytestmark = pytest.mark.gpu


def _kappa(factors):
    """Largest 2-norm condition number of V_n = Hadamard product of the
    Grams U_m^T U_m over m != n, over the modes n."""
    G = [u.T @ u for u in factors]
    ks = []
    for n in range(len(G)):
        V = np.ones_like(G[0])
        for m in range(len(G)):
            if m != n:
                V = V * G[m]
        ks.append(np.linalg.cond(V))
    return float(max(ks))


def test_small_uniform_fp64_matches_oracle():
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    U0 = synth.factors(cfg)
    at = make(dims, idx, vals)
    Ud = [dev(u.copy()) for u in U0]
    lam, fits = at.cpals(Ud, cfg["iters"])
    U, lam_o, fits_o, _ = oracle.cpals(dims, idx, vals, U0, cfg["iters"])
    print("fits gpu", fits, "oracle", fits_o)
    assert np.allclose(fits, fits_o, rtol=0, atol=1e-10)
    assert rel_err(lam.cpu().numpy(), lam_o) <= 1e-9
    for n in range(3):
        e = rel_err(Ud[n].cpu().numpy(), U[n])
        print("factor %d rel err %.3e" % (n, e))
        assert e <= 1e-9


@pytest.mark.parametrize("name,nnz", [("zipf3d-4Mx4Mx30k", 200_000), ("long5d-2^20x3-2^16x2", 200_000)])
def test_scaled_fp32_matches_oracle(name, nnz):
    cfg = synth.scaled(name, nnz=nnz, dims=None)
    # shrink the mode lengths so the oracle's dense Gram work stays small
    cfg["dims"] = tuple(min(d, 20_000) for d in cfg["dims"])
    dims, idx, vals = synth.tensor(cfg)
    U0 = synth.factors(cfg)
    at = make(dims, idx, vals)
    Ud = [dev(u.copy()) for u in U0]
    iters = 3
    lam, fits = at.cpals(Ud, iters)
    U, lam_o, fits_o, _ = oracle.cpals(dims, idx, vals, [u.astype(np.float64) for u in U0], iters)
    print(name, "fits gpu", fits, "oracle", fits_o)
    assert np.allclose(fits, fits_o, rtol=0, atol=1e-4)
    # FP32 factor storage, FP32 MTTKRP sums and the FP32-rounded inverse of
    # V perturb every least-squares update by a few FP32 units, which the
    # solve amplifies by the condition number of V (the Hadamard product of
    # the other modes' Grams): the bound is 100 kappa(V) 2^-24 over the Vs of
    # the initial and the final factors.
    kappa = max(_kappa([np.asarray(u, np.float64) for u in U0]), _kappa(U))
    tol = max(1e-5, 100.0 * kappa * 2.0 ** -24)
    for n in range(len(dims)):
        e = rel_err(Ud[n].cpu().numpy(), U[n])
        print("factor %d rel err %.3e (kappa(V) %.3e, bound %.3e)" % (n, e, kappa, tol))
        assert e <= tol


def test_bf16_factors_track_fp32():
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=200_000)
    cfg["dims"] = (20_000, 20_000, 3000)
    dims, idx, vals = synth.tensor(cfg)
    U0 = synth.factors(cfg)
    at = make(dims, idx, vals)
    Uf = [dev(u.copy()) for u in U0]
    _, fits32 = at.cpals(Uf, 3)
    Ub = [to_bf16_exact(u)[0] for u in U0]
    _, fitsb = at.cpals(Ub, 3)
    print("fp32", fits32, "bf16", fitsb)
    assert all(abs(a - b) < 2e-2 for a, b in zip(fits32, fitsb))


def test_exact_recovery_dense_low_rank():
    rng = np.random.default_rng(1)
    dims = (9, 8, 7)
    R = 3
    T = [rng.standard_normal((d, R)) for d in dims]
    X = np.einsum("ir,jr,kr->ijk", *T)
    cells = np.array(list(itertools.product(*[range(d) for d in dims])))
    idx = [cells[:, n].astype(np.uint32) for n in range(3)]
    vals = X[tuple(cells.T)]
    at = make(dims, idx, vals)
    Ud = [dev(t + 0.05 * rng.standard_normal(t.shape)) for t in T]
    lam, fits = at.cpals(Ud, 40)
    print("final fit", fits[-1])
    assert fits[-1] > 1 - 1e-6
    assert all(b >= a - 1e-9 for a, b in zip(fits, fits[1:]))


def test_singular_gram_reports_not_spd():
    from paper_2102_10245_gb300 import AltoError
    cfg = synth.CONFIGS["uniform3d-64x128x256"]
    dims, idx, vals = synth.tensor(cfg)
    U0 = synth.factors(cfg)
    U0[1][:, 3] = 0.0                 # zero column: V is singular
    at = make(dims, idx, vals)
    with pytest.raises(AltoError) as e:
        at.cpals([dev(u.copy()) for u in U0], 1)
    assert e.value.status == 6        # ALTO_ENOTSPD
    # the handle and the context stay usable
    lam, fits = at.cpals([dev(u.copy()) for u in synth.factors(cfg)], 1)
    assert np.isfinite(fits[0])


@pytest.mark.parametrize("R", [8, 24, 64])
@pytest.mark.parametrize("fdt", ["f64", "f32"])
def test_ranks_match_oracle(R, fdt):
    """Every update path: the fused one-pass update (R <= 32), the two-pass
    warp-row update (R = 64) and the generic one (other ranks)."""
    rng = np.random.default_rng(R)
    dims = (300, 200, 150)
    M = 20_000
    idx = [rng.integers(0, d, M).astype(np.uint32) for d in dims]
    vals = rng.random(M).astype(np.float64 if fdt == "f64" else np.float32)
    U0 = [rng.random((d, R)) for d in dims]
    at = make(dims, idx, vals)
    npdt = np.float64 if fdt == "f64" else np.float32
    Ud = [dev(u.astype(npdt)) for u in U0]
    iters = 4
    lam, fits = at.cpals(Ud, iters)
    U, lam_o, fits_o, _ = oracle.cpals(dims, idx, vals.astype(np.float64),
                                       [u.astype(npdt).astype(np.float64) for u in U0], iters)
    tol = 1e-9 if fdt == "f64" else 1e-3
    print(R, fdt, "fits gpu", fits, "oracle", fits_o)
    assert np.allclose(fits, fits_o, rtol=0, atol=tol * 10)
    assert rel_err(lam.cpu().numpy(), lam_o) <= tol
    for n in range(3):
        assert rel_err(Ud[n].cpu().numpy(), U[n]) <= tol


def test_bf16_values_match_oracle_on_rounded_values():
    """CP-ALS over a tensor whose values are stored as BF16 follows the FP64
    oracle run on the BF16-rounded values (the same bound as FP32 storage)."""
    from paper_2102_10245_gb300 import AltoTensor
    from helpers import dev_idx
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=200_000)
    cfg["dims"] = (20_000, 20_000, 3000)
    dims, idx, vals = synth.tensor(cfg)
    vb = torch.from_numpy(vals.astype(np.float32)).to(torch.bfloat16)
    vr = vb.to(torch.float64).numpy()
    U0 = synth.factors(cfg)
    at = AltoTensor(dims, dev_idx(idx), vb.cuda())
    Ud = [dev(u.copy()) for u in U0]
    iters = 3
    lam, fits = at.cpals(Ud, iters)
    U, lam_o, fits_o, _ = oracle.cpals(dims, idx, vr, [u.astype(np.float64) for u in U0], iters)
    print("bf16 values: fits gpu", fits, "oracle", fits_o)
    assert np.allclose(fits, fits_o, rtol=0, atol=1e-4)
    kappa = max(_kappa([np.asarray(u, np.float64) for u in U0]), _kappa(U))
    tol = max(1e-5, 100.0 * kappa * 2.0 ** -24)
    for n in range(len(dims)):
        e = rel_err(Ud[n].cpu().numpy(), U[n])
        print("factor %d rel err %.3e (bound %.3e)" % (n, e, tol))
        assert e <= tol
