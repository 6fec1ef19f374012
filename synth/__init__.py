"""Seeded synthetic sparse tensors shaped like the ALTO paper's workloads.

This package is shared by the tests, the benchmark, the oracle checks and
the CUDA library's callers.  It holds none of ALTO's arithmetic: it only
draws coordinates, values and factor matrices from seeded generators (numpy
for everything the oracle checks; torch's device generator for bulk timing
data) and removes duplicate coordinates.

Coordinate laws (stand-ins for the FROSTT / HaTen2 tensors of Table 1, which
are not available here):

* ``uniform``   -- every index uniform over its mode.
* ``zipf``      -- bounded Zipf(s) rank over {1..I_n} (inverse CDF by binary
  search in the cumulative table of k^-s, valid for any s > 0), mapped
  through a seeded random permutation of the mode so the heavy rows are
  spread over the index range.
* ``clustered`` -- Zipf-weighted cluster centres, each nonzero a uniform
  offset inside a box anchored at its centre.

Duplicate coordinates are removed and the draw is topped up until exactly M
distinct nonzeros remain; the surviving nonzeros are returned in random
order.  Indices are uint32 per mode (every configuration here has mode
lengths below 2^32).
"""
import math

import numpy as np
import torch

# ---------------------------------------------------------------------------
# named workloads

CONFIGS = {
    # 64 x 128 x 256, 20k distinct uniform nonzeros, FP64 values U(0,1),
    # rank 16 FP64 factors U(0,1), 5 CP-ALS iterations.
    "uniform3d-64x128x256": dict(
        dims=(64, 128, 256), nnz=20_000, laws=("uniform",) * 3,
        vals="uniform01", vdtype="f64", rank=16, fdist="uniform01",
        fdtype="f64", iters=5, seed=1),
    # 4M x 4M x 30k, 150M distinct nonzeros, Zipf(1.1) per mode over a
    # permutation, FP32 lognormal(0,1) values, rank 32 FP32 N(0,1) factors,
    # 10 CP-ALS iterations.
    "zipf3d-4Mx4Mx30k": dict(
        dims=(4_000_000, 4_000_000, 30_000), nnz=150_000_000,
        laws=(("zipf", 1.1),) * 3, vals="lognormal", vdtype="f32", rank=32,
        fdist="normal", fdtype="f32", iters=10, seed=2),
    # 12k x 60k x 5M x 100, 200M nonzeros in 50k Zipf(1.2)-weighted clusters
    # with offsets uniform in a 64^4 box, FP32 U(-1,1) values, rank 64.
    "clustered4d-12kx60kx5Mx100": dict(
        dims=(12_000, 60_000, 5_000_000, 100), nnz=200_000_000,
        laws=("clustered",), clusters=50_000, cluster_s=1.2, box=64,
        vals="uniform-11", vdtype="f32", rank=64, fdist="normal",
        fdtype="f32", iters=5, seed=3),
    # 2^20 x 2^20 x 2^20 x 2^16 x 2^16 (92 index bits), 60M nonzeros, modes
    # 0-2 uniform, modes 3-4 Zipf(0.9); FP32 U(0,1) values, rank 16.
    "long5d-2^20x3-2^16x2": dict(
        dims=(1 << 20, 1 << 20, 1 << 20, 1 << 16, 1 << 16), nnz=60_000_000,
        laws=("uniform", "uniform", "uniform", ("zipf", 0.9), ("zipf", 0.9)),
        vals="uniform01", vdtype="f32", rank=16, fdist="uniform01",
        fdtype="f32", iters=5, seed=4),
}


def scaled(name, nnz=None, dims=None, seed=None):
    """A copy of a named configuration with smaller nnz / dims / seed."""
    c = dict(CONFIGS[name])
    if nnz is not None:
        c["nnz"] = int(nnz)
    if dims is not None:
        c["dims"] = tuple(int(d) for d in dims)
    if seed is not None:
        c["seed"] = int(seed)
    return c


# ---------------------------------------------------------------------------
# laws


class BoundedZipf:
    """Zipf(s) ranks over {0..I-1} (rank 0 is the heaviest), any s > 0."""

    def __init__(self, I, s):
        w = np.arange(1, I + 1, dtype=np.float64) ** (-float(s))
        c = np.cumsum(w)
        self.cdf = torch.from_numpy(c / c[-1])
        self.I = I

    def draw(self, rng, n):
        """int64 torch tensor of n ranks."""
        u = torch.from_numpy(rng.random(n))
        r = torch.searchsorted(self.cdf, u, right=True)
        return r.clamp_(max=self.I - 1)


def _mode_sampler(rng, law, I):
    if law == "uniform":
        return lambda g, n: torch.from_numpy(g.integers(0, I, size=n, dtype=np.int64))
    if isinstance(law, tuple) and law[0] == "zipf":
        z = BoundedZipf(I, law[1])
        perm = torch.from_numpy(rng.permutation(I).astype(np.int64))
        return lambda g, n: perm[z.draw(g, n)]
    raise ValueError("unknown law %r" % (law,))


def _clustered_sampler(rng, dims, nclusters, s, box):
    """Centres uniform in [0, I_n - box_n], box_n = min(box, I_n); a nonzero
    picks a centre by a Zipf(s) weight and adds a uniform offset in the box."""
    N = len(dims)
    boxes = [min(box, d) for d in dims]
    centres = [torch.from_numpy(rng.integers(0, d - b + 1, size=nclusters, dtype=np.int64))
               for d, b in zip(dims, boxes)]
    z = BoundedZipf(nclusters, s)
    cperm = torch.from_numpy(rng.permutation(nclusters).astype(np.int64))

    def draw(g, n):
        c = cperm[z.draw(g, n)]
        return [centres[m][c] + torch.from_numpy(g.integers(0, boxes[m], size=n, dtype=np.int64))
                for m in range(N)]
    return draw


# ---------------------------------------------------------------------------
# dedup


def _radix_fits(dims):
    p = 1
    for d in dims:
        p *= int(d)
    return p <= (1 << 62)


def _linear(coords, dims):
    """Plain row-major linear index of each coordinate tuple (a dedup key)."""
    key = torch.zeros(coords[0].shape[0], dtype=torch.int64, device=coords[0].device)
    for c, d in zip(coords, dims):
        key.mul_(int(d)).add_(c)
    return key


def _unlinear(key, dims):
    out = [None] * len(dims)
    k = key.clone()
    for m in range(len(dims) - 1, -1, -1):
        d = int(dims[m])
        out[m] = torch.remainder(k, d)
        k = torch.div(k, d, rounding_mode="floor")
    return out


_M1 = -4658895280553007687   # 0xBF58476D1CE4E5B9 as int64
_M2 = -7723592293110705685   # 0x94D049BB133111EB as int64


def _mix64(x):
    """splitmix64 finaliser on int64 bit patterns (a dedup hash for index
    spaces above 2^62).  Logical right shifts are emulated with a mask."""
    def srl(v, s):
        return (v >> s) & ((1 << (64 - s)) - 1)
    x = x ^ srl(x, 30)
    x = x * _M1
    x = x ^ srl(x, 27)
    x = x * _M2
    return x ^ srl(x, 31)


def _hash(coords):
    h = torch.zeros(coords[0].shape[0], dtype=torch.int64, device=coords[0].device)
    for c in coords:
        h = _mix64(h ^ c)
    return h


def _sorted_unique(keys):
    s, _ = torch.sort(keys)
    if s.numel() == 0:
        return s
    keep = torch.ones(s.numel(), dtype=torch.bool, device=s.device)
    keep[1:] = s[1:] != s[:-1]
    return s[keep]


def _first_unique(h):
    """Indices of the first occurrence of every distinct value of h."""
    order = torch.sort(h, stable=True)[1]
    s = h[order]
    keep = torch.ones(s.numel(), dtype=torch.bool, device=s.device)
    keep[1:] = s[1:] != s[:-1]
    return order[keep]


def _distinct(draw, rng, dims, M):
    """Draw until M distinct coordinates exist; return them (uint32 numpy
    array per mode) in random order."""
    N = len(dims)
    cells = 1
    for d in dims:
        cells *= int(d)
    if M > cells:
        raise ValueError("nnz %d exceeds the %d cells of the tensor" % (M, cells))
    tg = torch.Generator().manual_seed(int(rng.integers(0, 1 << 62)))
    batch = max(1024, int(M * 1.15))
    if _radix_fits(dims):
        keys = torch.zeros(0, dtype=torch.int64)
        while keys.shape[0] < M:
            need = M - keys.shape[0]
            n = batch if keys.shape[0] == 0 else max(1024, int(need * 1.5))
            c = draw(rng, n)
            keys = _sorted_unique(torch.cat([keys, _linear(c, dims)]))
        sel = torch.randperm(keys.shape[0], generator=tg)[:M]
        coords = _unlinear(keys[sel], dims)
    else:
        coords = [torch.zeros(0, dtype=torch.int64) for _ in range(N)]
        h = torch.zeros(0, dtype=torch.int64)
        while coords[0].shape[0] < M:
            need = M - coords[0].shape[0]
            n = batch if coords[0].shape[0] == 0 else max(1024, int(need * 1.5))
            c = draw(rng, n)
            allc = [torch.cat([a, b]) for a, b in zip(coords, c)]
            allh = torch.cat([h, _hash(c)])
            first = _first_unique(allh)
            first, _ = torch.sort(first)
            coords = [a[first] for a in allc]
            h = allh[first]
        sel = torch.randperm(coords[0].shape[0], generator=tg)[:M]
        coords = [a[sel] for a in coords]
    return [c.to(torch.int32).numpy().view(np.uint32) for c in coords]


# ---------------------------------------------------------------------------
# public


def _values(rng, kind, M, dtype):
    if kind == "uniform01":
        v = rng.random(M)
    elif kind == "uniform-11":
        v = rng.random(M) * 2.0 - 1.0
    elif kind == "lognormal":
        v = rng.lognormal(0.0, 1.0, size=M)
    else:
        raise ValueError(kind)
    return v.astype(np.float64 if dtype == "f64" else np.float32)


def factors(cfg, seed_offset=1000):
    """Seeded initial factor matrices (I_n x R), in the configuration's
    factor dtype (FP64 or FP32).  Drawn in FP64 and rounded."""
    rng = np.random.default_rng(cfg["seed"] + seed_offset)
    R = cfg["rank"]
    out = []
    for d in cfg["dims"]:
        if cfg["fdist"] == "uniform01":
            f = rng.random((d, R))
        else:
            f = rng.standard_normal((d, R))
        out.append(f.astype(np.float64 if cfg["fdtype"] == "f64" else np.float32))
    return out


def tensor(cfg):
    """Return (dims, idx, vals): idx is a list of N uint32 arrays of length M
    and vals an FP64 or FP32 array, nonzeros distinct and in random order."""
    rng = np.random.default_rng(cfg["seed"])
    dims = tuple(int(d) for d in cfg["dims"])
    M = int(cfg["nnz"])
    laws = cfg["laws"]
    if laws and laws[0] == "clustered":
        draw = _clustered_sampler(rng, dims, cfg.get("clusters", 1024),
                                  cfg.get("cluster_s", 1.2), cfg.get("box", 64))
    else:
        samplers = [_mode_sampler(rng, law, d) for law, d in zip(laws, dims)]
        draw = lambda g, n: [s(g, n) for s in samplers]  # noqa: E731
    idx = _distinct(draw, rng, dims, M) if M > 0 else [np.zeros(0, np.uint32) for _ in dims]
    vals = _values(rng, cfg["vals"], M, cfg["vdtype"])
    return dims, idx, vals


def batch_config(seed):
    """One tensor of the batched workload: order U{3,4,5}; nnz log-uniform in
    [10k, 5M]; mode lengths log-uniform in [100, 10M]; law uniform, Zipf with
    s in [0.8, 1.5], or clustered; rank in {8, 16, 32, 64}; nnz clamped to
    half the cells."""
    rng = np.random.default_rng(10_000 + int(seed))
    N = int(rng.integers(3, 6))
    dims = tuple(int(round(math.exp(rng.uniform(math.log(100), math.log(1e7)))))
                 for _ in range(N))
    M = int(round(math.exp(rng.uniform(math.log(1e4), math.log(5e6)))))
    cells = 1
    for d in dims:
        cells *= d
    M = min(M, cells // 2)
    kind = int(rng.integers(0, 3))
    R = int(rng.choice([8, 16, 32, 64]))
    cfg = dict(dims=dims, nnz=M, vals="uniform01", vdtype="f32", rank=R,
               fdist="normal", fdtype="f32", iters=1, seed=20_000 + int(seed))
    if kind == 0:
        cfg["laws"] = ("uniform",) * N
    elif kind == 1:
        s = float(rng.uniform(0.8, 1.5))
        cfg["laws"] = (("zipf", s),) * N
    else:
        cfg["laws"] = ("clustered",)
        cfg["clusters"] = max(16, M // 4096)
        cfg["cluster_s"] = 1.2
        cfg["box"] = 64
    return cfg


# ---------------------------------------------------------------------------
# device-side generation (bulk timing data for variant selection)


def tensor_torch(cfg, device="cuda"):
    """The configuration's laws drawn with torch's generator on `device`
    (fast bulk generation for variant timing; not the numpy stream, so not
    for oracle parity).  Returns (dims, idx: list of int32 device tensors,
    vals: float32 device tensor), nonzeros distinct and in random order."""
    g = torch.Generator(device=device).manual_seed(int(cfg["seed"]))
    dims = tuple(int(d) for d in cfg["dims"])
    M = int(cfg["nnz"])
    N = len(dims)
    laws = cfg["laws"]

    def zipf_sampler(I, s):
        w = torch.arange(1, I + 1, dtype=torch.float64, device=device) ** (-float(s))
        cdf = torch.cumsum(w, 0)
        cdf /= cdf[-1].clone()
        return lambda n: torch.searchsorted(cdf, torch.rand(n, generator=g, dtype=torch.float64, device=device),
                                            right=True).clamp_(max=I - 1)

    if laws and laws[0] == "clustered":
        nc = int(cfg.get("clusters", 1024))
        boxes = [min(int(cfg.get("box", 64)), d) for d in dims]
        centres = [torch.randint(0, d - b + 1, (nc,), generator=g, device=device) for d, b in zip(dims, boxes)]
        z = zipf_sampler(nc, cfg.get("cluster_s", 1.2))
        cperm = torch.randperm(nc, generator=g, device=device)

        def draw(n):
            c = cperm[z(n)]
            return [centres[m][c] + torch.randint(0, boxes[m], (n,), generator=g, device=device) for m in range(N)]
    else:
        samplers = []
        for law, I in zip(laws, dims):
            if law == "uniform":
                samplers.append(lambda n, I=I: torch.randint(0, I, (n,), generator=g, device=device))
            else:
                zs = zipf_sampler(I, law[1])
                perm = torch.randperm(I, generator=g, device=device)
                samplers.append(lambda n, zs=zs, perm=perm: perm[zs(n)])

        def draw(n):
            return [smp(n) for smp in samplers]

    batch = max(1024, int(M * 1.15))
    if _radix_fits(dims):
        keys = torch.zeros(0, dtype=torch.int64, device=device)
        while keys.shape[0] < M:
            need = M - keys.shape[0]
            n = batch if keys.shape[0] == 0 else max(1024, int(need * 1.5))
            keys = _sorted_unique(torch.cat([keys, _linear(draw(n), dims)]))
        sel = torch.randperm(keys.shape[0], generator=g, device=device)[:M]
        coords = _unlinear(keys[sel], dims)
    else:
        coords = [torch.zeros(0, dtype=torch.int64, device=device) for _ in range(N)]
        h = torch.zeros(0, dtype=torch.int64, device=device)
        while coords[0].shape[0] < M:
            need = M - coords[0].shape[0]
            n = batch if coords[0].shape[0] == 0 else max(1024, int(need * 1.5))
            c = draw(n)
            allc = [torch.cat([a, b]) for a, b in zip(coords, c)]
            allh = torch.cat([h, _hash(c)])
            first, _ = torch.sort(_first_unique(allh))
            coords = [a[first] for a in allc]
            h = allh[first]
        sel = torch.randperm(coords[0].shape[0], generator=g, device=device)[:M]
        coords = [a[sel] for a in coords]
    vals = torch.rand(M, generator=g, device=device, dtype=torch.float32)
    return dims, [c.to(torch.int32) for c in coords], vals


def factors_torch(cfg, device="cuda", dtype=torch.float32, seed_offset=1000):
    """N(0,1) factor matrices drawn on `device`."""
    g = torch.Generator(device=device).manual_seed(int(cfg["seed"]) + seed_offset)
    return [torch.randn(d, cfg["rank"], generator=g, device=device).to(dtype) for d in cfg["dims"]]
