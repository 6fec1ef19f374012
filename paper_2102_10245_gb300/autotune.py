"""Variant selection for MTTKRP: the autotuner (times every accumulation
variant of a (tensor, mode) on the GPU and keeps the fastest), the cheap
per-mode statistics a learned predictor reads, the predictor itself (an MLP
trained and run by libalto's nn kernels), and the regret bookkeeping that
compares a set of picks with the autotuned ones.

The accumulation strategies are the ones of Sec. 3.3 (direct atomic updates
for low fiber reuse, buffered accumulation for high reuse) in their GPU
forms: ATOMIC, WARPAGG (register runs + replicated hot rows) and SMEM
(shared-memory Temp over the unit's output interval), each with a choice of
the segment count L of Sec. 3.2.  The library's own
rule (alto_resolve_variant with AUTO) is the method without the predictor.
"""
import math

import numpy as np
import torch

from .alto import BF16, F32, F64, VAR_ATOMIC, VAR_SMEM, VAR_WARPAGG, AltoTensor
from .mlp import MLP

# The autotuner's choices for one (tensor, mode): accumulation variant x
# segment count of the ALTO line (Sec. 3.2 leaves L free; the GPU kernels use
# it to cut the line into thread-block units), the count as a factor of the
# tensor's own L (alto_set_parts; SMEM keeps L, it reads the segments'
# intervals).  VARIANTS / PARTS are the two columns.
CANDIDATES = ((VAR_ATOMIC, 1.0), (VAR_WARPAGG, 1.0), (VAR_SMEM, 1.0),
              (VAR_ATOMIC, 0.25), (VAR_WARPAGG, 0.25), (VAR_ATOMIC, 4.0), (VAR_WARPAGG, 4.0))
VARIANTS = tuple(v for v, _ in CANDIDATES)
PARTS = tuple(f for _, f in CANDIDATES)
_NAMES = {VAR_ATOMIC: "atomic", VAR_WARPAGG: "warpagg", VAR_SMEM: "smem"}
VARIANT_LABELS = tuple("%s/L%s" % (_NAMES[v], "" if f == 1.0 else ("*%g" % f)) for v, f in CANDIDATES)


def parts_for(at, factor):
    """Segment count of candidate factor ``factor`` on tensor ``at`` (0 for the
    tensor's own L)."""
    if factor == 1.0:
        return 0
    L = int(at.stats()["nparts"])
    return max(1, min(int(round(L * factor)), max(at.nnz, 1)))


def apply(at, mode, k):
    """Set mode ``mode`` of ``at`` to candidate ``k`` (variant and segment
    count), for alto_mttkrp calls and batches planned afterwards."""
    at.set_variant(mode, VARIANTS[k])
    at.set_parts(mode, parts_for(at, PARTS[k]))

FEATURES = (
    "order", "log2_len", "log2_nnz", "log2_reuse", "log2_rank", "distinct_frac", "hot_share",
    "log2_hot_rows", "log2_unit_width_p50", "log2_unit_width_p90", "unit_fit_smem", "log2_max_interval",
    "mean_log2_other_len", "key_words", "log2_gather_bytes",
)

SMEM_TEMP_BYTES = 96 * 1024  # shared Temp budget of the SMEM variant per block


def _torch_dtype(fdtype):
    return {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[fdtype]


def features(at, mode, rank, fdtype=BF16):
    """Cheap statistics of one (tensor, mode), all known after alto_create:
    order, lengths, nnz, fiber reuse, rank, distinct output rows, hot-row
    mass, thread-block unit interval widths and the share of units whose
    output interval fits the shared buffer."""
    I, D, reuse, maxivl, hot_n, hot_share, w50, w90 = at.mode_stats(mode)
    fsz = {F64: 8, F32: 4, BF16: 2}[fdtype]
    osz = 8 if fdtype == F64 else 4
    rows = min(SMEM_TEMP_BYTES // (rank * osz), int(I))
    others = [at.dims[m] for m in range(at.N) if m != mode]
    gather = sum(others) * rank * fsz
    return np.array([
        at.N, math.log2(I), math.log2(max(at.nnz, 1)), math.log2(max(reuse, 1e-6)), math.log2(rank),
        D / I, hot_share, math.log2(hot_n + 1), math.log2(w50 + 1), math.log2(w90 + 1),
        at.unit_fit(mode, rows), math.log2(maxivl + 1),
        float(np.mean(np.log2(others))) if others else 0.0, at.layout()["key_words"], math.log2(gather + 1),
    ], dtype=np.float64)


def time_variants(at, mode, factors, out, candidates=None, target_ms=0.25, max_reps=64, trials=2):
    """Device time (ms) of one MTTKRP call per candidate (indices into
    CANDIDATES; all by default).  Each candidate's calls are captured ``reps``
    times into one CUDA graph, so launch overhead of the host does not enter;
    the best of ``trials`` replays counts.  Leaves the mode on the automatic
    variant and the tensor's own L."""
    res = []
    stream = torch.cuda.Stream()
    for k in (range(len(CANDIDATES)) if candidates is None else candidates):
        apply(at, mode, k)
        at.mttkrp(mode, factors, out, stream=stream)  # allocates the hot-row replicas
        stream.synchronize()
        # estimate one call to size the graph
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        at.mttkrp(mode, factors, out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        est = max(e0.elapsed_time(e1), 1e-3)
        reps = int(min(max_reps, max(2, math.ceil(target_ms / est))))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            g.capture_begin(capture_error_mode="thread_local")
            try:
                for _ in range(reps):
                    at.mttkrp(mode, factors, out, stream=stream)
            finally:
                g.capture_end()
        best = float("inf")
        with torch.cuda.stream(stream):
            g.replay()
            for _ in range(trials):
                e0.record(stream)
                g.replay()
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / reps)
        del g
        res.append(best)
    at.set_variant(mode, 0)
    at.set_parts(mode, 0)
    return np.array(res)


def rule_pick(at, mode, rank, fdtype=BF16):
    """Index into CANDIDATES of the library's built-in choice (its variant
    with the tensor's own L)."""
    v = at.resolve_variant(mode, rank, fdtype)
    return CANDIDATES.index((v, 1.0)) if (v, 1.0) in CANDIDATES else CANDIDATES.index((VAR_WARPAGG, 1.0))


def make_item(cfg, device="cuda", fdtype=BF16):
    """An ALTO tensor and factors for one synthetic configuration, generated
    on the device."""
    import synth
    dims, idx, vals = synth.tensor_torch(cfg, device)
    at = AltoTensor(dims, idx, vals)
    del idx, vals
    factors = synth.factors_torch(cfg, device, _torch_dtype(fdtype))
    return at, factors


def collect(seeds, device="cuda", fdtype=BF16, log=None):
    """Autotuner timings for every mode of every seeded batch configuration:
    features (K x F), times (K x V ms), the rule's pick (K), and the
    (seed, mode, nnz) of each row."""
    import synth
    feats, times, rule, meta = [], [], [], []
    for k, seed in enumerate(seeds):
        cfg = synth.batch_config(seed)
        at, factors = make_item(cfg, device, fdtype)
        R = cfg["rank"]
        odt = torch.float64 if fdtype == F64 else torch.float32
        for mode in range(at.N):
            out = torch.empty((at.dims[mode], R), dtype=odt, device=device)
            feats.append(features(at, mode, R, fdtype))
            times.append(time_variants(at, mode, factors, out))
            rule.append(rule_pick(at, mode, R, fdtype))
            meta.append((seed, mode, at.nnz))
            del out
        at.close()
        del factors
        if log and (k % 100 == 0 or k == len(seeds) - 1):
            log("collected %d / %d tensors" % (k + 1, len(seeds)))
    return dict(features=np.array(feats), times=np.array(times), rule=np.array(rule, np.int64),
                meta=np.array(meta, np.int64), feature_names=np.array(FEATURES),
                variants=np.array(VARIANTS, np.int64), parts=np.array(PARTS, np.float64))


def regret(times, picks):
    """(total, mean) regret of ``picks`` against the fastest variant:
    total = sum of picked times / sum of best times - 1 (what a batch of all
    these calls loses), mean = average of per-call ratios - 1."""
    times = np.asarray(times, np.float64)
    picked = times[np.arange(len(times)), np.asarray(picks)]
    best = times.min(axis=1)
    return float(picked.sum() / best.sum() - 1.0), float(np.mean(picked / best) - 1.0)


def targets(times):
    """Training targets: log2 of each variant's time over the row's best."""
    t = np.asarray(times, np.float64)
    return np.log2(t / t.min(axis=1, keepdims=True))


class Predictor:
    """MLP features -> relative log-time per variant; the pick is the
    smallest prediction.  Standardisation constants are taken from the
    training features."""

    def __init__(self, hidden=(64, 64), seed=0, device="cuda"):
        self.hidden = tuple(hidden)
        self.seed = seed
        self.device = device
        self.net = None
        self.mu = self.sd = None

    def _x(self, feats):
        x = (np.asarray(feats, np.float64) - self.mu) / self.sd
        return torch.from_numpy(x.astype(np.float32)).to(self.device)

    def fit(self, feats, times, epochs=2000, lr=3e-3, weight=None):
        feats = np.asarray(feats, np.float64)
        self.mu = feats.mean(axis=0)
        self.sd = feats.std(axis=0) + 1e-6
        X = self._x(feats)
        Y = torch.from_numpy(targets(times).astype(np.float32)).to(self.device)
        mask = None
        if weight is not None:
            w = np.repeat(np.asarray(weight, np.float64)[:, None], Y.shape[1], axis=1)
            mask = torch.from_numpy((w / w.mean()).astype(np.float32)).to(self.device)
        self.net = MLP((feats.shape[1],) + self.hidden + (Y.shape[1],), seed=self.seed, device=self.device)
        return self.net.fit(X, Y, mask=mask, epochs=epochs, lr=lr)

    def scores(self, feats):
        return self.net.predict(self._x(feats)).cpu().numpy()

    def pick(self, feats):
        return self.scores(feats).argmin(axis=1)

    def configure(self, at, rank, fdtype=BF16):
        """Set every mode of ``at`` to the predicted candidate (variant and
        segment count), so plain alto_mttkrp / alto_cpals calls use it;
        returns the variants."""
        feats = np.array([features(at, n, rank, fdtype) for n in range(at.N)])
        picks = [int(p) for p in self.pick(feats)]
        for n, k in enumerate(picks):
            apply(at, n, k)
        return [VARIANTS[k] for k in picks]

    def save(self, path):
        arrays = {"mu": self.mu, "sd": self.sd, "hidden": np.array(self.hidden)}
        for i, (W, b) in enumerate(self.net.params):
            arrays["W%d" % i] = W.cpu().numpy()
            arrays["b%d" % i] = b.cpu().numpy()
        np.savez(path, **arrays)

    @classmethod
    def load(cls, path, device="cuda"):
        d = np.load(path)
        p = cls(hidden=tuple(int(h) for h in d["hidden"]), device=device)
        p.mu, p.sd = d["mu"], d["sd"]
        sizes = [d["W0"].shape[1]] + [d["W%d" % i].shape[0] for i in range(len(p.hidden) + 1)]
        p.net = MLP(sizes, device=device)
        for i, pr in enumerate(p.net.params):
            pr[0].copy_(torch.from_numpy(d["W%d" % i]))
            pr[1].copy_(torch.from_numpy(d["b%d" % i]))
        return p

    def choose(self, feats, measure=None, margin=0.0):
        """Picks with the autotuner as fallback: rows whose two best
        predictions are within ``margin`` (log2 units) are timed by
        ``measure(row) -> times`` instead."""
        s = self.scores(feats)
        picks = s.argmin(axis=1)
        if measure is not None and margin > 0:
            srt = np.sort(s, axis=1)
            for r in np.flatnonzero(srt[:, 1] - srt[:, 0] < margin):
                picks[r] = int(np.argmin(measure(r)))
        return picks


def _seed_range(text):
    a, b = text.split(":")
    return list(range(int(a), int(b)))


def main(argv=None):
    """Collect autotuner timings on the GPU and store them (numpy .npz):
    python -m paper_2102_10245_gb300.autotune --train 0:2000 --heldout 100000:100256 --out FILE"""
    import argparse
    import sys
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", default="0:2000")
    ap.add_argument("--heldout", default="100000:100256")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    log = lambda m: print("[autotune %.0fs] %s" % (time.time() - t0, m), file=sys.stderr, flush=True)  # noqa: E731
    t0 = time.time()
    from .build import kernel_source_hash
    dev_name = torch.cuda.get_device_name()
    parts = {"device": np.array(dev_name), "kernel_hash": np.array(kernel_source_hash()),
             "candidates": np.array(VARIANT_LABELS)}
    for name, text in (("heldout", a.heldout), ("train", a.train)):
        seeds = _seed_range(text)
        chunks = []
        for c0 in range(0, len(seeds), 250):   # saved after every chunk
            chunks.append(collect(seeds[c0:c0 + 250], log=log))
            for k in chunks[0]:
                vals = [c[k] for c in chunks]
                parts["%s_%s" % (name, k)] = vals[0] if k in ("feature_names", "variants", "parts") else np.concatenate(vals)
            np.savez_compressed(a.out, **parts)
            log("%s: %d / %d tensors saved" % (name, min(c0 + 250, len(seeds)), len(seeds)))


if __name__ == "__main__":
    main()
