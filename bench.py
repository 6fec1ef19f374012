"""Benchmark of the ALTO hot path on GB300.

One step = the whole hot path over one synthetic tensor: ALTO generation
(linearization, ordering, value permutation, partitioning, intervals, stats,
flags) followed by the configuration's CP-ALS iterations, each an all-mode
MTTKRP sweep plus the per-mode CP-ALS update.  The headline value is the
all-mode MTTKRP nonzero throughput of that whole job,
    value = iters * N * nnz / step time   [Gnnz/s],
with the inputs resident in HBM when the timed region starts.  The MTTKRP
kernels alone are also timed (CUDA events recorded by the library around
every MTTKRP launch inside the timed steps) and reported against the HBM
roofline of their compulsory bytes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica of the workload (weak
scaling; the path needs no exchange between GPUs); rank 0 prints the line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "all-mode MTTKRP Gnnz/s + % HBM roofline; CP-ALS s/iter vs plain FP32"
DEFAULT_CONFIG = "zipf3d-4Mx4Mx30k"
FALLBACK_HBM_GBS = 6800.0
CPU_SAMPLE_NNZ = 40_000_000      # oracle CPU-baseline sample, all host threads
CPU_SAMPLE_NNZ_1T = 10_000_000   # the same, one thread (about 8-10 s)
GEN_SAMPLE_NNZ = 10_000_000      # oracle generation sample (encode + sort)
TRANSPOSE_SAMPLE_NNZ = 10_000_000  # oracle transposition sample (stable sorts by coordinates)


def TRANSPOSE_MODES(N):
    """The transposition the bench times: the last mode first, then the
    others in order (for 4M x 4M x 30k: the 30k-long mode leads)."""
    return [N - 1] + list(range(N - 1))
RANKSPEC_NNZ = 20_000_000        # rank-specialisation comparison tensor
REF_STEP_NNZ = 4_000_000         # reference-arm step sample


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default=DEFAULT_CONFIG)
    p.add_argument("--fdtype", default=None, choices=[None, "f32", "bf16", "f64"])
    p.add_argument("--variant", type=int, default=0, help="force one MTTKRP variant for every mode")
    p.add_argument("--nparts", default="0", help="line segments L (0 = automatic); --mttkrp-only: comma list")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-bf16", action="store_true", help="skip the BF16-factor CP-ALS comparison")
    p.add_argument("--no-rankspec", action="store_true", help="skip the rank-specialisation comparison")
    p.add_argument("--no-transpose", action="store_true", help="skip the transposition measurement")
    p.add_argument("--no-batched", action="store_true", help="skip the batched + learned sub-measurement")
    p.add_argument("--sub-batch-items", type=int, default=64,
                   help="held-out batched tensors in the default line's batched sub-measurement")
    p.add_argument("--nnz", type=int, default=0,
                   help="profiling only: the workload's generator with fewer nonzeros")
    p.add_argument("--mttkrp-only", action="store_true",
                   help="time alto_mttkrp per mode and variant instead of the full step")
    p.add_argument("--variants", default="0", help="--mttkrp-only: comma-separated variants (0 = auto)")
    p.add_argument("--modes", default="", help="--mttkrp-only: comma-separated modes (default all)")
    p.add_argument("--reps", type=int, default=3, help="--mttkrp-only: timed calls per (variant, mode)")
    p.add_argument("--batch-items", type=int, default=256, help="batched workload: held-out tensors")
    p.add_argument("--train-items", type=int, default=2000, help="batched workload: training tensors")
    p.add_argument("--err-items", type=int, default=8, help="batched workload: tensors checked against FP64")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU, replicas)

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        return self.parse(self.lines)

    @staticmethod
    def parse(lines):
        """Median SM clock, maximum clock and the throttle reasons seen in
        nvidia-smi CSV lines (the FIELDS order, no header, no units)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# helpers

def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    """Hash of the MTTKRP kernel sources (a recorded ncu traffic figure or
    timing set is only used while it matches)."""
    import paper_2102_10245_gb300.build as lb
    return lb.kernel_source_hash()


def recorded_traffic(config, fdtype, calls):
    """DRAM bytes per MTTKRP launch (averaged over the timed launches' modes)
    from a committed ncu summary, if it was taken on the current kernel
    source (else None)."""
    p = os.path.join(ROOT, "profiles", "mttkrp_dram_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get("%s/%s" % (config, fdtype))
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    per = e.get("bytes_per_launch", {})
    tot = sum(int(calls[n]) for n in range(len(calls)))
    if tot == 0 or any(str(n) not in per for n in range(len(calls))):
        return None
    return sum(per[str(n)] * int(calls[n]) for n in range(len(calls))) / tot


def mttkrp_bytes(nnz, key_bytes, val_bytes, distinct, R, fbytes, obytes, n):
    """Compulsory bytes of one mode-n MTTKRP: the key and value stream, every
    distinct input-factor row once and every distinct output row once."""
    N = len(distinct)
    b = nnz * (key_bytes + val_bytes)
    b += sum(distinct[m] * R * fbytes for m in range(N) if m != n)
    b += distinct[n] * R * obytes
    return b


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)

def oracle_sweep_time(dims, idx, vals, U64, nnz_sample):
    import oracle
    sidx = [a[:nnz_sample] for a in idx]
    sv = np.asarray(vals[:nnz_sample], dtype=np.float64)
    t0 = time.perf_counter()
    for n in range(len(dims)):
        oracle.mttkrp(dims, sidx, sv, U64, n)
    return time.perf_counter() - t0


def oracle_sweep_time_threads(dims, idx, vals, U64, nnz_sample, threads):
    """The oracle's all-mode MTTKRP on `threads` host threads (each owns the
    output rows i_n mod T; bit-identical to the single-thread sums).
    Returns (seconds, threads used)."""
    import oracle
    sidx = [a[:nnz_sample] for a in idx]
    sv = np.asarray(vals[:nnz_sample], dtype=np.float64)
    used = 1
    t0 = time.perf_counter()
    for n in range(len(dims)):
        _, used = oracle.mttkrp_threads(dims, sidx, sv, U64, n, threads)
    return time.perf_counter() - t0, used


def oracle_generation_time(dims, idx, nnz_sample):
    """The oracle's linearization and ordering (bit-loop encode, stable sort
    by key with an index tie-break) on one host thread; seconds."""
    import oracle
    sidx = [a[:nnz_sample] for a in idx]
    t0 = time.perf_counter()
    keys = oracle.encode(dims, sidx)
    oracle.sort_perm(keys)
    return time.perf_counter() - t0


def oracle_transpose_time(idx, modes, nnz_sample):
    """The oracle's transposition sort (one stable sort per chosen mode, by
    coordinate) of the first nnz_sample nonzeros on one host thread; seconds."""
    import oracle
    coords = np.stack([np.asarray(a[:nnz_sample], dtype=np.int64) for a in idx], 1)
    t0 = time.perf_counter()
    oracle.transpose_order(coords, modes)
    return time.perf_counter() - t0


def host_cpu():
    """Host CPU model and logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = synth.CONFIGS[args.config]
    dims, idx, vals = synth.tensor(cfg)
    U64 = [u.astype(np.float64) for u in synth.factors(cfg)]
    S = min(REF_STEP_NNZ, len(vals))
    N = len(dims)
    for _ in range(args.warmup):
        oracle_sweep_time(dims, idx, vals, U64, S)
    ts = [oracle_sweep_time(dims, idx, vals, U64, S) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    value = N * S / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gnnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "dims": list(dims), "nnz": len(vals), "rank": cfg["rank"],
                   "sample_nnz": S, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "Gnnz/s", "cores": 1, "kind": "oracle",
                         "sample": "all-mode FP64 COO MTTKRP over the first %d of %d nonzeros per step"
                                   % (S, len(vals))},
        "e2e": {"value": value, "unit": "Gnnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm

def run_ours(args, rank, world, local):
    from paper_2102_10245_gb300 import AltoTensor, launch_count, torch_allocator, GRAM_AUTO, GRAM_CUDA_CORES
    import paper_2102_10245_gb300.build as lb
    lb.build()

    cfg = synth.CONFIGS[args.config]
    fdtype = args.fdtype or cfg["fdtype"]
    dims, idx, vals = synth.tensor(cfg)
    U0 = synth.factors(cfg)
    N, M, R, iters = len(dims), len(vals), cfg["rank"], cfg["iters"]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[fdtype]
    vdt = torch.float64 if fdtype == "f64" else torch.float32

    # CPU baseline first (rank 0, single GPU only), before any GPU work
    cpu = None
    gen_oracle = None
    tr_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S = min(CPU_SAMPLE_NNZ, M)
        U64 = [u.astype(np.float64) for u in U0]
        hc = host_cpu()
        nth = max(1, int(hc["nproc"] or 1))
        tm, used = oracle_sweep_time_threads(dims, idx, vals, U64, S, nth)
        t1 = oracle_sweep_time(dims, idx, vals, U64, min(S, CPU_SAMPLE_NNZ_1T))
        S1 = min(S, CPU_SAMPLE_NNZ_1T)
        cpu = {"value": N * S / tm / 1e9, "unit": "Gnnz/s", "cores": used, "kind": "oracle",
               "cpu": hc["model"], "nproc": hc["nproc"],
               "sample": "all-mode FP64 COO MTTKRP (the oracle) over the first %d of %d nonzeros on %d host "
                         "threads (output rows split by thread, bit-identical sums), %.1f s" % (S, M, used, tm),
               "single_thread": {"value": N * S1 / t1 / 1e9, "unit": "Gnnz/s", "cores": 1,
                                 "sample": "the same on one thread over the first %d nonzeros, %.1f s" % (S1, t1)}}
        SG = min(GEN_SAMPLE_NNZ, M)
        tg = oracle_generation_time(dims, idx, SG)
        gen_oracle = {"gnnz_s": SG / tg / 1e9, "cores": 1, "seconds": tg,
                      "sample": "oracle encode (bit loops) + stable sort (qsort, index tie-break) of the first "
                                "%d nonzeros, one thread" % SG}
        del U64
        if not args.no_transpose:
            ST = min(TRANSPOSE_SAMPLE_NNZ, M)
            tt = oracle_transpose_time(idx, TRANSPOSE_MODES(N), ST)
            tr_oracle = {"gnnz_s": ST / tt / 1e9, "cores": 1, "seconds": tt,
                         "sample": "oracle transposition sort (one stable numpy argsort per mode, modes %s) of the "
                                   "first %d nonzeros, one thread" % (TRANSPOSE_MODES(N), ST)}

    dev = torch.device("cuda", torch.cuda.current_device())
    # inputs resident in HBM
    idx_d = [torch.from_numpy(a.view(np.int32)).to(dev) for a in idx]
    vals_d = torch.from_numpy(vals.astype(np.float64 if fdtype == "f64" else np.float32)).to(dev)
    U0_d = [torch.from_numpy(u).to(dev).to(tdt) for u in U0]
    Uw = [torch.empty_like(u) for u in U0_d]
    lam = torch.empty(R, dtype=torch.float64, device=dev)
    alloc = torch_allocator()
    variants = [args.variant] * N if args.variant else None
    stream = torch.cuda.current_stream()

    stats = {}
    prof_ms = np.zeros(N)
    prof_calls = np.zeros(N, dtype=np.int64)
    phase = []   # (create_start, create_end / cpals_start, cpals_end) events per timed step

    def step(record):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)] if record else None
        if record:
            evs[0].record(stream)
        at = AltoTensor(dims, idx_d, vals_d, allocator=alloc, variants=variants, nparts=int(args.nparts))
        if record:
            at.profile(True)
        for w, u in zip(Uw, U0_d):
            w.copy_(u)
        if record:
            evs[1].record(stream)
        _, fits = at.cpals(Uw, iters, lam=lam)
        if record:
            evs[2].record(stream)
            phase.append(evs)
            ms, calls = at.profile_read()
            prof_ms[:] += ms
            prof_calls[:] += calls
        if not stats:
            stats.update(at.stats())
            stats["key_words"] = at.layout()["key_words"]
            stats["key_bytes"] = at.key_bytes()
            stats["fits"] = fits
        at.close()
        return fits

    # warm-up
    for _ in range(max(args.warmup, 0)):
        step(False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    n0 = launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        fits = step(True)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - n0
    clk = clocks.stop()
    barrier(world)
    create_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in phase)
    cpals_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in phase)
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    units = sum_over_ranks(float(iters * N * M), world)
    value = units / (ms_step / 1e3) / 1e9

    # MTTKRP kernels against the HBM roofline
    fb = {"f32": 4, "bf16": 2, "f64": 8}[fdtype]
    ob = 8 if fdtype == "f64" else 4
    vb = 8 if fdtype == "f64" else 4
    kb = stats["key_bytes"]
    per_mode_bytes = [mttkrp_bytes(M, kb, vb, stats["distinct"], R, fb, ob, n) for n in range(N)]
    tot_bytes = sum(per_mode_bytes[n] * prof_calls[n] for n in range(N))
    tot_ms = float(prof_ms.sum())
    achieved = tot_bytes / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else 0.0
    peak, peak_src = measured_peak()
    sweep_ms = tot_ms / max(1, int(prof_calls.min()))
    traffic = recorded_traffic(args.config, fdtype, prof_calls) if not args.nnz else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                "kernel": "alto MTTKRP (all modes, incl. output zeroing)",
                "bytes_per_launch": {str(n): int(per_mode_bytes[n]) for n in range(N)}}

    # CP-ALS seconds per iteration and MTTKRP sweep time with BF16 factor
    # storage, and with BF16 values plus BF16 factors, against the plain FP32
    # form (the same iterations, creation excluded)
    precision = None
    if fdtype == "f32" and not args.no_bf16:
        at32 = AltoTensor(dims, idx_d, vals_d, allocator=alloc, variants=variants, nparts=int(args.nparts))
        at16 = AltoTensor(dims, idx_d, vals_d.to(torch.bfloat16), allocator=alloc, variants=variants,
                          nparts=int(args.nparts))
        res = {}
        for name, at_, dt, eng in (("f32", at32, torch.float32, GRAM_AUTO), ("bf16", at32, torch.bfloat16, GRAM_AUTO),
                                   ("bf16_cuda_core_gram", at32, torch.bfloat16, GRAM_CUDA_CORES),
                                   ("bf16_values", at16, torch.bfloat16, GRAM_AUTO)):
            at_.set_gram_engine(eng)
            U = [u.to(dt) for u in U0_d]
            W = [torch.empty_like(u) for u in U]
            for w, u in zip(W, U):
                w.copy_(u)
            at_.cpals(W, 2, lam=lam)  # warm-up
            at_.profile(True)
            at_.profile_read()
            reps, tot, fl = 3, 0.0, None
            for _ in range(reps):
                for w, u in zip(W, U):
                    w.copy_(u)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, fl = at_.cpals(W, iters, lam=lam)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            pms, pcalls = at_.profile_read()
            at_.profile(False)
            res[name] = (tot / reps / 1e3 / iters, fl[-1] if fl else None,
                         float(np.sum(pms)) / max(1, int(np.min(pcalls))))
            del U, W
        at32.close()
        at16.close()
        precision = {"f32_s_per_iter": res["f32"][0], "bf16_s_per_iter": res["bf16"][0],
                     "bf16_cuda_core_gram_s_per_iter": res["bf16_cuda_core_gram"][0],
                     "bf16_values_s_per_iter": res["bf16_values"][0],
                     "bf16_speedup": res["f32"][0] / res["bf16"][0],
                     "bf16_values_speedup": res["f32"][0] / res["bf16_values"][0],
                     "mttkrp_sweep_ms": {k: v[2] for k, v in res.items()},
                     "fit_f32": res["f32"][1], "fit_bf16": res["bf16"][1], "fit_bf16_values": res["bf16_values"][1],
                     "note": "CP-ALS only (MTTKRP sweeps + updates), one created tensor per value dtype, 3 timed "
                             "runs; bf16 = BF16 factor storage (Gram matrices on the tensor cores), "
                             "bf16_cuda_core_gram = the same with the CUDA-core Gram, bf16_values = BF16 values and "
                             "BF16 factors, FP32 accumulation throughout"}

    # rank specialisation (Sec. 4.5): the rank- and order-specialised fused
    # kernel against the runtime-rank generic kernel, on a smaller tensor
    # of the same generator, every mode, FP32 factors
    rankspec = None
    if not args.no_rankspec:
        rcfg = synth.scaled(args.config, nnz=min(RANKSPEC_NNZ, M))
        rdims, ridx, rvals = synth.tensor_torch(rcfg, dev)
        at = AltoTensor(rdims, ridx, rvals, allocator=alloc)
        del ridx
        res = {}
        for Rr in (8, 16, 32, 64):
            U = synth.factors_torch(dict(rcfg, rank=Rr), dev, torch.float32)
            outs = [torch.empty(d, Rr, dtype=torch.float32, device=dev) for d in rdims]
            t = {}
            for name, var in (("specialised", 0), ("generic", 5)):
                for n in range(N):
                    at.set_variant(n, var)
                sweep = lambda: [at.mttkrp(n, U, out=outs[n]) for n in range(N)]  # noqa: E731
                sweep()
                t[name] = _time_k(sweep, 3, stream)
            res[str(Rr)] = {"specialised_ms": t["specialised"], "generic_ms": t["generic"],
                            "ratio": t["generic"] / t["specialised"]}
            del U, outs
        at.close()
        rankspec = {"nnz": int(len(rvals)), "per_rank": res,
                    "what": "all-mode MTTKRP sweep, FP32 factors: specialised (order and rank fixed at compile "
                            "time, fused body) vs generic (runtime order and rank, scalar atomics)"}

    # sparse tensor transposition (Sec. 5) by partial radix sort: every mode
    # (the full reordering) and the leading mode alone, from the ALTO tensor
    # to the transposed COO (input positions, coordinates, values) in HBM
    transpose = None
    if not args.no_transpose:
        at = AltoTensor(dims, idx_d, vals_d, allocator=alloc)
        lay = at.layout()
        res = {}
        for name, modes in (("all_modes", TRANSPOSE_MODES(N)), ("leading_mode", TRANSPOSE_MODES(N)[:1])):
            nb = sum(lay["bits"][m] for m in modes)
            fn = lambda: at.transpose(modes)  # noqa: E731
            fn()
            ms = _time_k(fn, 3, stream)
            res[name] = {"modes": modes, "key_bits": nb, "radix_passes": -(-max(nb, 1) // 8), "ms": ms,
                         "gnnz_s": M / (ms / 1e3) / 1e9}
        at.close()
        transpose = dict(res, oracle=tr_oracle, index_bits=sum(lay["bits"]),
                         what="alto_transpose: sort key cut from the stored index, stable LSD radix sort over the "
                              "chosen modes' bits only, gather of input positions, coordinates (int64) and values")

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        idx_h = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in idx]
        vals_h = vals_d.cpu().pin_memory()
        U0_h = [u.cpu().pin_memory() for u in U0_d]
        out_h = [torch.empty(u.shape, dtype=u.dtype).pin_memory() for u in U0_d]
        lam_h = torch.empty(R, dtype=torch.float64).pin_memory()
        h2d = sum(a.numel() * a.element_size() for a in idx_h) + vals_h.numel() * vals_h.element_size() \
            + sum(u.numel() * u.element_size() for u in U0_h)
        d2h = sum(u.numel() * u.element_size() for u in out_h) + R * 8 + iters * 8

        def step_e2e():
            at = AltoTensor(dims, idx_h, vals_h, allocator=alloc, variants=variants, nparts=int(args.nparts))
            for w, u in zip(Uw, U0_h):
                w.copy_(u, non_blocking=True)
            _, f = at.cpals(Uw, iters, lam=lam)
            for o, w in zip(out_h, Uw):
                o.copy_(w, non_blocking=True)
            lam_h.copy_(lam, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            at.close()
            return f
        step_e2e()
        k2 = max(2, args.steps // 2)
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k2):
            step_e2e()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / k2, world)
        e2e = {"value": units / (ms_e2e / 1e3) / 1e9, "unit": "Gnnz/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e2e, "steps": k2}

    batched = None
    if not args.no_batched:
        sub = run_batched(args, rank, world, local, n_items=args.sub_batch_items, steps=3, emit=False)
        if sub is not None:
            batched = {k: sub[k] for k in ("value", "unit", "ms_per_step", "config", "plain_fp32",
                                           "speedup_vs_plain_fp32", "speedup_vs_fp32_batched", "context",
                                           "predictor", "rel_err_vs_fp64",
                                           "batch", "roofline")}
            batched["form"] = "BF16 factors, every (tensor, mode) in one graph, predictor picks"

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "Gnnz/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": fdtype, "data": "synthetic",
        "config": {"workload": args.config, "dims": list(dims), "nnz": M, "rank": R, "iters": iters,
                   "step": "alto_create + %d CP-ALS iterations (all-mode MTTKRP + update)" % iters,
                   "l2": "inputs larger than L2 (COO %.1f GB, ALTO stream %.1f GB)"
                         % ((N * 4 + vb) * M / 1e9, (kb + vb) * M / 1e9),
                   "variant": stats["variant"] if args.variant == 0 else [args.variant] * N},
        "mttkrp": {"sweep_ms": sweep_ms, "gnnz_s": N * M / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None,
                   "ms_per_mode": [float(prof_ms[n] / max(1, prof_calls[n])) for n in range(N)],
                   "calls": [int(c) for c in prof_calls]},
        "create_ms": create_ms,
        "generation": {"gnnz_s": M / (create_ms / 1e3) / 1e9, "ms": create_ms,
                       "what": "alto_create from HBM-resident COO: encode, radix sort, value permutation, "
                               "partition and intervals, statistics, flags",
                       "oracle": gen_oracle},
        "cpals_s_per_iter": cpals_ms / 1e3 / iters,
        "cpals_precision": precision,
        "rank_specialisation": rankspec,
        "transpose": transpose,
        "batched": batched,
        "fit_last": fits[-1] if fits else None,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


BATCH_CONFIG = "batched-256"
BATCH_HELDOUT = 100_000          # seeds of the held-out batched tensors
TIMINGS = os.path.join(ROOT, "paper_2102_10245_gb300", "data", "variant_timings.npz")


def _time_k(fn, k, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def run_batched(args, rank, world, local, n_items=None, steps=None, emit=True):
    """The batched + learned workload: all-mode MTTKRP of 256 seeded tensors
    of order 3-5 (nnz 10k-5M, lengths 100-10M, uniform / Zipf / clustered,
    R in {8, 16, 32, 64}).  Headline: BF16 factors, every (tensor, mode) in
    one graph-captured batch, variants picked by the MLP trained on the
    autotuner timings of 2,000 other seeded tensors.  Beside it: the plain
    FP32 form (one alto_mttkrp call per tensor and mode, built-in rule) and
    the predictor's regret against the autotuned picks of these tensors."""
    from paper_2102_10245_gb300 import AltoTensor, Batch, launch_count
    from paper_2102_10245_gb300 import autotune as tune
    import paper_2102_10245_gb300.build as lb
    lb.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    K, W = (steps or args.steps), max(args.warmup, 0)
    log = lambda m: print("[batched %.0fs] %s" % (time.time() - t_start, m), file=sys.stderr, flush=True)  # noqa
    t_start = time.time()

    seeds = list(range(BATCH_HELDOUT, BATCH_HELDOUT + (n_items or args.batch_items)))
    cfgs = [synth.batch_config(s) for s in seeds]
    tensors = []
    for cfg in cfgs:
        dims, idx, vals = synth.tensor_torch(cfg, dev)
        tensors.append(AltoTensor(dims, idx, vals))
        del idx, vals
    work = sum(at.nnz * at.N for at in tensors)
    log("created %d tensors, %.1f M nonzeros" % (len(tensors), sum(at.nnz for at in tensors) / 1e6))

    # plain FP32: one call per (tensor, mode), the built-in variant rule
    f32 = [synth.factors_torch(cfg, dev, torch.float32) for cfg in cfgs]
    outs = [[torch.empty(d, cfg["rank"], dtype=torch.float32, device=dev) for d in cfg["dims"]] for cfg in cfgs]

    def plain():
        for at, U, O in zip(tensors, f32, outs):
            for n in range(at.N):
                at.mttkrp(n, U, out=O[n])
    for _ in range(W):
        plain()
    torch.cuda.synchronize()
    ms_plain = _time_k(plain, K, stream)
    items32 = [(at, n, U, O[n]) for at, U, O in zip(tensors, f32, outs) for n in range(at.N)]
    b32 = Batch(items32)
    for _ in range(W):
        b32.run()
    ms_b32_rule = _time_k(b32.run, K, stream)
    b32.close()
    del b32, items32
    log("plain FP32 %.2f ms, FP32 batched (rule) %.2f ms" % (ms_plain, ms_b32_rule))

    # BF16 factors (the same values rounded), FP32 copies released one by one
    bf = []
    for U in f32:
        bf.append([u.to(torch.bfloat16) for u in U])
        U.clear()
    del f32
    torch.cuda.empty_cache()
    items = [(at, n, U, O[n]) for at, U, O in zip(tensors, bf, outs) for n in range(at.N)]
    feats = np.array([tune.features(at, n, U[0].shape[1]) for at, n, U, _ in items])
    rule = np.array([tune.rule_pick(at, n, U[0].shape[1]) for at, n, U, _ in items])

    # the predictor: trained on the GPU by libalto's nn kernels
    timing_set = None
    if os.path.exists(TIMINGS):
        d = np.load(TIMINGS)
        tr_f, tr_t, src = d["train_features"], d["train_times"], os.path.relpath(TIMINGS, ROOT)
        stored = str(d["kernel_hash"]) if "kernel_hash" in d.files else None
        timing_set = {"file": src, "kernel_hash": stored, "kernel_hash_now": kernel_source_hash(),
                      "current": stored == kernel_source_hash(), "candidates": int(tr_t.shape[1])}
        if not timing_set["current"]:
            log("warning: the stored timing set was measured on other MTTKRP kernel sources")
        if tr_t.shape[1] != len(tune.CANDIDATES):
            raise RuntimeError("stored timing set has %d candidates, the autotuner %d: re-collect it with "
                               "python -m paper_2102_10245_gb300.autotune" % (tr_t.shape[1], len(tune.CANDIDATES)))
    else:
        log("no stored timings: collecting the training set now")
        d = tune.collect(range(0, args.train_items), log=log)
        tr_f, tr_t, src = d["features"], d["times"], "collected in this run"
    pred = tune.Predictor(seed=0)
    t0 = time.perf_counter()
    losses = pred.fit(tr_f, tr_t)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    picks = pred.pick(feats)
    infer_ms = (time.perf_counter() - t0) * 1e3
    log("predictor trained in %.1f s (loss %.4f -> %.4f)" % (train_s, losses[0], losses[-1]))

    # the autotuner on the held-out items: the judge of the predictor
    times = np.array([tune.time_variants(at, n, U, O) for at, n, U, O in items])
    best = times.argmin(axis=1)
    reg_mlp = tune.regret(times, picks)
    reg_rule = tune.regret(times, rule)
    log("regret: predictor %.3f / %.3f, rule %.3f / %.3f" % (reg_mlp + reg_rule))

    def plan(sel):
        """A batch whose items run the chosen candidates' accumulation
        variants with each tensor's own segment count: the autotuner's finer
        segment counts win in a call of their own, but inside one persistent
        launch over many items a short unit leaves each warp too few chunks to
        fill its pipeline (measured slower)."""
        return Batch(items, variants=[tune.VARIANTS[int(k)] for k in sel])

    def batch_ms(sel):
        b = plan(sel)
        for _ in range(W):
            b.run()
        ms = _time_k(b.run, K, stream)
        info = b.info()
        b.close()
        return ms, info
    ms_rule, _ = batch_ms(rule)
    ms_best, _ = batch_ms(best)
    bh = plan(picks)
    for _ in range(W):
        bh.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    n0 = launch_count()
    torch.cuda.nvtx.range_push("bf16_batched_learned")  # lets a profiler select this region
    ms = _time_k(bh.run, K, stream)
    torch.cuda.nvtx.range_pop()
    launches = launch_count() - n0
    clk = clocks.stop()
    info = bh.info()

    # error of the BF16 batch against FP64 on the smallest tensors: the
    # reference is libalto's FP64 MTTKRP of the same tensor with the FP32
    # factors widened to FP64 (that path matches the CPU oracle to 1e-12 in
    # the parity tests; the bench itself does not run the oracle here)
    errs = []
    small = sorted(range(len(tensors)), key=lambda i: tensors[i].nnz)[:args.err_items]
    bh.run()
    torch.cuda.synchronize()
    for i in small:
        cfg = cfgs[i]
        dims, idx, vals = synth.tensor_torch(cfg, dev)
        at64 = AltoTensor(dims, idx, vals.to(torch.float64))
        U64 = [u.to(torch.float64) for u in synth.factors_torch(cfg, dev, torch.float32)]
        for n in range(len(dims)):
            ref = at64.mttkrp(n, U64)
            got = outs[i][n].to(torch.float64)
            errs.append(float(torch.linalg.norm(got - ref) / max(float(torch.linalg.norm(ref)), 1e-300)))
        at64.close()
        del idx, vals
    bh.close()

    # roofline of the batch: compulsory bytes of every item over the graph time
    tot_bytes = 0
    for at, n, U, _ in items:
        st = at.stats()
        kb = at.key_bytes()
        tot_bytes += mttkrp_bytes(at.nnz, kb, 4, st["distinct"], U[0].shape[1], 2, 4, n)
    peak, peak_src = measured_peak()
    achieved = tot_bytes / (ms / 1e3) / 1e9
    value = work / (ms / 1e3) / 1e9
    if rank != 0:
        return None
    lab = tune.VARIANT_LABELS
    line = {
        "metric": METRIC, "value": value, "unit": "Gnnz/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "%s: all-mode MTTKRP of %d seeded tensors (order 3-5, nnz 10k-5M log-uniform, "
                               "lengths 100-10M, uniform/Zipf/clustered, R in {8,16,32,64})"
                               % (BATCH_CONFIG, len(tensors)),
                   "nnz_total": int(sum(at.nnz for at in tensors)), "items": len(items),
                   "step": "one graph replay: every (tensor, mode) MTTKRP, BF16 factors, FP32 accumulation",
                   "l2": "inputs larger than L2 (%.1f GB of keys and values)"
                         % (sum(at.nnz for at in tensors) * 12 / 1e9)},
        "plain_fp32": {"ms": ms_plain, "gnnz_s": work / (ms_plain / 1e3) / 1e9,
                       "form": "one alto_mttkrp call per (tensor, mode), FP32 factors, built-in variant rule"},
        "speedup_vs_plain_fp32": ms_plain / ms,
        "speedup_vs_fp32_batched": ms_b32_rule / ms,
        "context": {"fp32_batched_rule_ms": ms_b32_rule, "bf16_batched_rule_ms": ms_rule,
                    "bf16_batched_autotuned_ms": ms_best},
        "predictor": {"train": src, "timing_set": timing_set, "train_rows": int(len(tr_f)), "train_s": train_s,
                      "infer_ms": infer_ms,
                      "loss_first_last": [losses[0], losses[-1]],
                      "regret_total": reg_mlp[0], "regret_mean": reg_mlp[1],
                      "rule_regret_total": reg_rule[0], "rule_regret_mean": reg_rule[1],
                      "picks": {lab[v]: int((picks == v).sum()) for v in range(len(lab))},
                      "autotuned": {lab[v]: int((best == v).sum()) for v in range(len(lab))}},
        "rel_err_vs_fp64": {"max": max(errs) if errs else None, "items": len(errs),
                            "sample": "every mode of the %d smallest tensors" % len(small),
                            "reference": "libalto FP64 MTTKRP, FP32 factors widened to FP64"},
        "batch": info,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": peak_src,
                     "kernel": "the whole batch graph (group kernels, hot-row reduce, output zeroing)"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_mttkrp_only(args):
    """Time alto_mttkrp per (variant, mode) on one created tensor; one JSON
    line per (variant, mode).  Used for kernel profiling."""
    from paper_2102_10245_gb300 import AltoTensor, torch_allocator
    import paper_2102_10245_gb300.build as lb
    lb.build()
    cfg = synth.scaled(args.config, nnz=args.nnz) if args.nnz else synth.CONFIGS[args.config]
    fdtype = args.fdtype or cfg["fdtype"]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[fdtype]
    dims, idx, vals = synth.tensor(cfg)
    U = synth.factors(cfg)
    dev = torch.device("cuda", torch.cuda.current_device())
    idx_d = [torch.from_numpy(a.view(np.int32)).to(dev) for a in idx]
    vals_d = torch.from_numpy(vals.astype(np.float64 if fdtype == "f64" else np.float32)).to(dev)
    Ud = [torch.from_numpy(u).to(dev).to(tdt) for u in U]
    modes = [int(m) for m in args.modes.split(",")] if args.modes else list(range(len(dims)))
    for v, L in [(int(x), int(y)) for x in args.variants.split(",") for y in args.nparts.split(",")]:
        at = AltoTensor(dims, idx_d, vals_d, allocator=torch_allocator(), nparts=L)
        for n in modes:
            at.set_variant(n, v)
            out = at.mttkrp(n, Ud)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.reps):
                at.mttkrp(n, Ud, out=out)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.reps
            print(json.dumps({"workload": args.config, "nnz": len(vals), "dtype": fdtype, "variant": v,
                              "nparts": at.stats()["nparts"], "mode": n, "ms": ms,
                              "gnnz_s": len(vals) / ms / 1e6}), flush=True)
        at.close()


def main():
    args = parse()
    if args.mttkrp_only:
        torch.cuda.set_device(0)
        run_mttkrp_only(args)
        return
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == BATCH_CONFIG:
        run_batched(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
