"""The batched workload at its real sizes against the oracle.

The held-out batched tensors (order 3-5, nnz up to 5M, mode lengths up to
10M, uniform / Zipf / clustered coordinates, rank 8-64) run uncapped in one
graph-captured batch with BF16 factors and FP32 accumulation, with the
library's automatic variants (so the hot-row tables of the skewed tensors are
active).  Every mode of the 8 tensors with the most nonzeros and of the 8 most
skewed Zipf tensors is compared with the oracle on up to 10k sampled output
rows: within 1e-5 of the oracle run on the BF16-rounded factors (what the GPU
multiplies; the rest is FP32 accumulation order) and within 1e-2 of the
oracle run on the unrounded FP32 factors (the BF16 rounding itself).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import make, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HELDOUT = range(100_000, 100_256)
SAMPLE_ROWS = 10_000


def _selected():
    cfgs = {s: synth.batch_config(s) for s in HELDOUT}
    largest = sorted(cfgs, key=lambda s: -cfgs[s]["nnz"])[:8]
    zipf = [s for s in cfgs if isinstance(cfgs[s]["laws"][0], tuple) and s not in largest]
    skewed = sorted(zipf, key=lambda s: -cfgs[s]["laws"][0][1])[:8]
    return [cfgs[s] for s in largest + skewed]


def test_batched_heldout_real_size_matches_oracle(alto_lib):
    from paper_2102_10245_gb300 import Batch
    cfgs = _selected()
    rng = np.random.default_rng(11)
    items, keep, refs = [], [], []
    for cfg in cfgs:
        dims, idx, vals = synth.tensor(cfg)
        at = make(dims, idx, vals)
        U32 = synth.factors_torch(cfg, "cuda", torch.float32)
        U16 = [u.to(torch.bfloat16) for u in U32]
        outs = [torch.full((d, cfg["rank"]), float("nan"), dtype=torch.float32, device="cuda") for d in dims]
        for n in range(len(dims)):
            items.append((at, n, U16, outs[n]))
        keep.append((at, U32, U16, outs))
        refs.append((cfg, dims, idx, vals, U32, U16, outs))
    b = Batch(items)
    b.run()
    torch.cuda.synchronize()
    hot_modes = 0
    worst_r, worst_u = 0.0, 0.0
    for cfg, dims, idx, vals, U32, U16, outs in refs:
        at = next(k[0] for k in keep if k[3] is outs)
        for n in range(len(dims)):
            hot_modes += int(at.mode_stats(n)[4] > 0)
            used = np.unique(idx[n])
            rows = np.sort(rng.choice(used, size=min(SAMPLE_ROWS, len(used)), replace=False)).astype(np.int64)
            got = outs[n][torch.from_numpy(rows).cuda()].to(torch.float64).cpu().numpy()

            def fetch(U):
                return lambda m, ids: U[m][torch.from_numpy(ids).cuda()].to(torch.float64).cpu().numpy()
            ref_r = oracle.mttkrp_sampled(dims, idx, vals, fetch(U16), n, rows)
            ref_u = oracle.mttkrp_sampled(dims, idx, vals, fetch(U32), n, rows)
            er, eu = rel_err(got, ref_r), rel_err(got, ref_u)
            worst_r, worst_u = max(worst_r, er), max(worst_u, eu)
            assert er <= 1e-5, (cfg["seed"], dims, n, er)
            assert eu <= 1e-2, (cfg["seed"], dims, n, eu)
    print("batched real size: %d tensors, %d items, %d modes with hot rows, worst rel err %.2e (rounded "
          "factors) %.2e (unrounded)" % (len(refs), len(items), hot_modes, worst_r, worst_u))
    assert hot_modes > 0
    b.close()
