"""Plain FP64 CPU oracle for the ALTO hot path (Helal et al., ICS '21).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of ``bench.py`` may import this package; the product path never does.
It shares no code with the CUDA library; the only thing both sides use is
the seeded input generator package ``synth``.

What each function follows in the paper:

* ``bit_map`` / ``encode`` / ``decode`` -- Sec. 3.1 (Fig. 2 text, Eq. 1):
  one key bit at a time, levels from the LSB, shortest mode first inside a
  level, ties by mode index.  Implemented in C (``alto_oracle.c``) as
  explicit bit loops.
* ``sort_perm`` -- Sec. 3.1 ordering stage: ascending key, ties in input
  order (C ``qsort`` with an index tie-break).
* ``partition`` / ``intervals`` -- Sec. 3.2: ``floor(l*M/L)`` boundaries and
  tight per-mode [min, max] intervals.
* ``flags`` -- Sec. 3.3 last paragraph: internal element = its row along the
  mode is touched by exactly one segment.
* ``mttkrp`` -- Sec. 2.2 definition, Alg. 1 in COO form: direct FP64
  summation in input order.  ``mttkrp_threads`` splits the same sums over
  host threads by output row (bit-identical; used to time the oracle on
  all host cores).
* ``cpals`` -- Sec. 2.2 CPD-ALS; the paper defers its conventions to
  SPLATT / Tensor Toolbox, so this is the Kolda-Bader CP-ALS: per mode,
  MTTKRP, Hadamard product of the other Gram matrices, Cholesky solve,
  column normalisation (2-norm in the first iteration, max(1, max|.|) after),
  and the fit from ||X||, lambda and the last mode's MTTKRP.
* ``compression_ratio`` (Eq. 2), ``sfc_bits`` (Eq. 3), ``use_buffered``
  (Sec. 3.3 conflict rule: reuse = M / I_n, buffered iff reuse > 4).
* ``transpose_order`` / ``transpose`` -- Sec. 5 sparse tensor transposition,
  which reduces to sorting the nonzeros by their coordinates in the new mode
  order: starting from ALTO order (``encode`` + ``sort_perm``), one stable
  sort per chosen mode, least significant first, so ties keep ALTO order.

Parity pins for every function live in ``tests/test_oracle.py``.  The CP-ALS
equality with SPLATT claimed in Sec. 4.1 is parity unpinned: neither SPLATT
nor Tensor Toolbox is available to compare against.
"""
import ctypes
import math

import numpy as np

from . import build as _build

_MAXB = 128
_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        lib.orc_bit_map.argtypes = [i32, P, P, P]
        lib.orc_encode.argtypes = [i32, P, i64, P, i32, P]
        lib.orc_decode.argtypes = [i32, P, i64, P, P]
        lib.orc_sort_perm.argtypes = [i64, P, P]
        lib.orc_partition.argtypes = [i64, i64, P]
        lib.orc_intervals.argtypes = [i32, i64, P, i64, P, P]
        lib.orc_flags.argtypes = [i32, ctypes.c_uint64, i32, i64, P, i64, P, P]
        lib.orc_mttkrp.argtypes = [i32, P, i64, P, i32, P, P, i32, i32, P, P]
        lib.orc_mttkrp_threads.argtypes = [i32, P, i64, P, i32, P, P, i32, i32, P, i32]
        for f in (lib.orc_bit_map, lib.orc_encode, lib.orc_decode,
                  lib.orc_sort_perm, lib.orc_partition, lib.orc_intervals,
                  lib.orc_flags, lib.orc_mttkrp, lib.orc_mttkrp_threads):
            f.restype = i32
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.uint64))


def _idx_arrays(idx):
    """Per-mode index arrays as contiguous uint32 or int64 plus their width."""
    arrs = []
    width = 4
    for a in idx:
        a = np.asarray(a)
        if a.dtype not in (np.uint32, np.int64):
            a = a.astype(np.int64)
        arrs.append(a)
    if any(a.dtype == np.int64 for a in arrs):
        arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in arrs]
        width = 8
    else:
        arrs = [np.ascontiguousarray(a) for a in arrs]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arrs, ptrs, width


def bits_per_mode(dims):
    """Eq. 1 with whole bits: b_n = ceil(log2 I_n); I_n = 1 needs 0 bits."""
    return [int(max(0, int(d) - 1).bit_length()) for d in dims]


def bit_map(dims):
    """Return (nbits[N], pos[N][128], B): pos[n][l] = key bit of bit l of i_n."""
    lib = _load()
    d = _dims(dims)
    N = len(d)
    nbits = np.zeros(N, dtype=np.int32)
    pos = np.zeros((N, _MAXB), dtype=np.int32)
    B = lib.orc_bit_map(N, _ptr(d), _ptr(nbits), _ptr(pos))
    if B < 0:
        raise ValueError("bad dims %r" % (dims,))
    return nbits, pos, B


def encode(dims, idx):
    """ALTO keys of the nonzeros in input order, as an (M, 2) uint64 array of
    (lo, hi) words."""
    lib = _load()
    d = _dims(dims)
    arrs, ptrs, width = _idx_arrays(idx)
    M = len(arrs[0]) if arrs else 0
    keys = np.zeros((M, 2), dtype=np.uint64)
    rc = lib.orc_encode(len(d), _ptr(d), M, ptrs, width, _ptr(keys))
    if rc != 0:
        raise ValueError("index out of range in mode %d" % (-rc - 1))
    return keys


def decode(dims, keys):
    """Inverse of ``encode``: (M, N) uint64 coordinates."""
    lib = _load()
    d = _dims(dims)
    keys = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    M = keys.shape[0]
    out = np.zeros((M, len(d)), dtype=np.uint64)
    lib.orc_decode(len(d), _ptr(d), M, _ptr(keys), _ptr(out))
    return out


def sort_perm(keys):
    """perm[i] = input position of the i-th nonzero in ascending key order,
    equal keys in input order."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    M = keys.shape[0]
    perm = np.zeros(M, dtype=np.int64)
    lib.orc_sort_perm(M, _ptr(keys), _ptr(perm))
    return perm


def partition(M, L):
    """Segment boundaries floor(l*M/L), l = 0..L (Sec. 3.2)."""
    lib = _load()
    bounds = np.zeros(L + 1, dtype=np.int64)
    if lib.orc_partition(M, L, _ptr(bounds)) != 0:
        raise ValueError("L must be >= 1")
    return bounds


def intervals(coords_sorted, bounds):
    """(L, N, 2) uint64 closed intervals [start, end] per segment and mode."""
    lib = _load()
    c = np.ascontiguousarray(coords_sorted, dtype=np.uint64)
    M, N = c.shape
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    L = len(b) - 1
    ivl = np.zeros((L, N, 2), dtype=np.uint64)
    lib.orc_intervals(N, M, _ptr(c), L, _ptr(b), _ptr(ivl))
    return ivl


def flags(coords_sorted, In, n, bounds):
    """uint8 per element in ALTO order: 1 = internal (row touched by one
    segment only), 0 = boundary."""
    lib = _load()
    c = np.ascontiguousarray(coords_sorted, dtype=np.uint64)
    M, N = c.shape
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    out = np.zeros(M, dtype=np.uint8)
    if lib.orc_flags(N, int(In), n, M, _ptr(c), len(b) - 1, _ptr(b), _ptr(out)) != 0:
        raise MemoryError("oracle flags")
    return out


def mttkrp(dims, idx, vals, factors, mode, rows=None):
    """Mode-``mode`` MTTKRP by direct FP64 summation (Sec. 2.2, Alg. 1).

    ``factors[m]`` is I_m x R; ``factors[mode]`` is ignored (may be None).
    ``rows``: optional iterable of output rows; only those are accumulated
    (the others stay zero) -- used to check large tensors on sampled rows.
    Returns an I_mode x R float64 array.
    """
    lib = _load()
    d = _dims(dims)
    N = len(d)
    arrs, ptrs, width = _idx_arrays(idx)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    M = v.shape[0]
    R = None
    fs = []
    for m in range(N):
        if m == mode or factors[m] is None:
            fs.append(None)
            continue
        f = np.ascontiguousarray(factors[m], dtype=np.float64)
        R = f.shape[1]
        fs.append(f)
    if R is None:  # order-1 tensor: no other factor; R from the mode's own
        R = np.asarray(factors[mode]).shape[1]
    fptrs = (ctypes.c_void_p * N)(*[(f.ctypes.data if f is not None else 0) for f in fs])
    out = np.zeros((int(d[mode]), R), dtype=np.float64)
    mask = None
    if rows is not None:
        mask = np.zeros(int(d[mode]), dtype=np.uint8)
        mask[np.asarray(rows, dtype=np.int64)] = 1
    lib.orc_mttkrp(N, _ptr(d), M, ptrs, width, _ptr(v), fptrs, R, mode,
                   _ptr(mask) if mask is not None else None, _ptr(out))
    return out


def mttkrp_threads(dims, idx, vals, factors, mode, threads):
    """``mttkrp`` on ``threads`` host threads (each owns the output rows
    i_n mod T and sums their nonzeros in input order, so the result is
    bit-identical to ``mttkrp``).  Returns (out, threads used)."""
    lib = _load()
    d = _dims(dims)
    N = len(d)
    arrs, ptrs, width = _idx_arrays(idx)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    fs = [None if (m == mode or factors[m] is None) else np.ascontiguousarray(factors[m], dtype=np.float64)
          for m in range(N)]
    R = next(f.shape[1] for f in fs if f is not None)
    fptrs = (ctypes.c_void_p * N)(*[(f.ctypes.data if f is not None else 0) for f in fs])
    out = np.zeros((int(d[mode]), R), dtype=np.float64)
    used = lib.orc_mttkrp_threads(N, _ptr(d), v.shape[0], ptrs, width, _ptr(v), fptrs, R, mode, _ptr(out),
                                  int(threads))
    return out, used


def mttkrp_sampled(dims, idx, vals, get_rows, mode, rows):
    """Rows ``rows`` (sorted, distinct) of the mode-``mode`` MTTKRP by its
    definition, without the full factor matrices: only the nonzeros whose
    output row is in ``rows`` contribute, so they are kept, every input mode
    is relabeled to the distinct rows those nonzeros touch, and ``mttkrp``
    runs on that small problem (a relabeling of rows changes no sum).
    ``get_rows(m, ids)`` returns the FP64 rows ``ids`` of factor m.  Returns a
    len(rows) x R array in the order of ``rows``."""
    rows = np.asarray(rows, dtype=np.int64)
    out_idx = np.asarray(idx[mode]).astype(np.int64)
    keep = np.isin(out_idx, rows)
    sub_idx, sub_dims, fac = [], [], []
    for m in range(len(dims)):
        a = np.asarray(idx[m]).astype(np.int64)[keep]
        if m == mode:
            sub_idx.append(np.searchsorted(rows, a).astype(np.int64))
            sub_dims.append(len(rows))
            fac.append(None)
        else:
            u, inv = np.unique(a, return_inverse=True)
            sub_idx.append(inv.astype(np.int64))
            sub_dims.append(max(len(u), 1))
            f = np.asarray(get_rows(m, u), dtype=np.float64)
            if len(u) == 0:
                f = np.zeros((1, f.shape[1] if f.ndim == 2 and f.shape[1] else 1))
            fac.append(f)
    v = np.asarray(vals, dtype=np.float64)[keep]
    R = next(f.shape[1] for f in fac if f is not None)
    fac[mode] = np.zeros((1, R))
    return mttkrp(sub_dims, sub_idx, v, fac, mode)


def transpose_order(coords, modes):
    """Sec. 5 transposition as a sort by coordinates.  ``coords`` is M x N,
    rows in ALTO order; returns the positions (into those rows) of the
    nonzeros in the lexicographic order of columns modes[0], modes[1], ...
    (modes[0] most significant), ties in the given order.  One stable
    ``argsort`` per chosen mode, the last chosen mode first."""
    coords = np.asarray(coords)
    order = np.arange(coords.shape[0], dtype=np.int64)
    for m in reversed([int(x) for x in modes]):
        order = order[np.argsort(coords[order, m], kind="stable")]
    return order


def transpose(dims, idx, modes):
    """Transposition of the COO tensor (dims, idx) by ``modes``: returns
    (order, src) -- the ALTO positions and the input positions of the
    nonzeros in transposed order.  ALTO order comes from ``encode`` and
    ``sort_perm``; duplicates therefore keep input order."""
    keys = encode(dims, idx)
    alto = sort_perm(keys)
    M = len(alto)
    coords = np.zeros((M, len(dims)), dtype=np.int64)
    for n, a in enumerate(idx):
        coords[:, n] = np.asarray(a, dtype=np.int64)[alto]
    order = transpose_order(coords, modes)
    return order, alto[order]


def reuse(dims, M):
    """Average fiber reuse per mode, M / I_n (Sec. 3.3)."""
    return [M / float(d) for d in dims]


def use_buffered(dims, M):
    """Sec. 3.3 conflict rule: buffered (local Temp + pull reduction) iff the
    reuse is more than the 4 memory operations of the buffered path."""
    return [r > 4.0 for r in reuse(dims, M)]


def compression_ratio(dims, Wb):
    """Eq. 2: sum_n ceil(log2 I_n / Wb) / ceil(sum_n log2 I_n / Wb)."""
    b = bits_per_mode(dims)
    return sum(math.ceil(x / Wb) for x in b) / math.ceil(sum(b) / Wb)


def sfc_bits(dims):
    """Eq. 3 per nonzero: N * max_n log2 I_n bits (Z-Morton index)."""
    return len(dims) * max(bits_per_mode(dims))


def norm_sq(dims, idx, vals):
    """||X||_F^2 of the tensor whose entry at a coordinate is the sum of the
    values of all nonzeros at that coordinate (duplicates add up, as in the
    MTTKRP of Alg. 1)."""
    v = np.asarray(vals, dtype=np.float64)
    if v.shape[0] == 0:
        return 0.0
    c = np.stack([np.asarray(i, dtype=np.int64) for i in idx], axis=1)
    order = np.lexsort(c.T[::-1])
    cs = c[order]
    start = np.ones(len(cs), dtype=bool)
    start[1:] = (cs[1:] != cs[:-1]).any(axis=1)
    sums = np.add.reduceat(v[order], np.flatnonzero(start))
    return float(np.dot(sums, sums))


def cpals(dims, idx, vals, factors0, iters):
    """Kolda-Bader CP-ALS in FP64 (Sec. 2.2), fixed iteration count.

    Returns (factors, lam, fits, mttkrp_last) where fits[t] is the fit after
    iteration t.
    """
    import scipy.linalg

    N = len(dims)
    U = [np.array(f, dtype=np.float64, copy=True) for f in factors0]
    R = U[0].shape[1]
    v = np.asarray(vals, dtype=np.float64)
    normX2 = norm_sq(dims, idx, v)
    G = [u.T @ u for u in U]
    lam = np.ones(R)
    fits = []
    Mlast = None
    for it in range(iters):
        for n in range(N):
            Mn = mttkrp(dims, idx, v, U, n)
            V = np.ones((R, R))
            for m in range(N):
                if m != n:
                    V = V * G[m]
            c = scipy.linalg.cho_factor(V, lower=True)
            Unew = scipy.linalg.cho_solve(c, Mn.T).T
            if it == 0:
                lam = np.sqrt(np.sum(Unew * Unew, axis=0))
            else:
                lam = np.maximum(np.max(np.abs(Unew), axis=0), 1.0)
            Unew = Unew / lam
            U[n] = Unew
            G[n] = Unew.T @ Unew
            Mlast = Mn
        V = np.ones((R, R))
        for m in range(N):
            V = V * G[m]
        normP2 = float(lam @ V @ lam)
        iprod = float(np.sum(np.sum(U[N - 1] * Mlast, axis=0) * lam))
        resid = math.sqrt(max(0.0, normX2 + normP2 - 2.0 * iprod))
        fits.append(1.0 - resid / math.sqrt(normX2))
    return U, lam, fits, Mlast
