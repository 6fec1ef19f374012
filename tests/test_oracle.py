"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
worked example printed in the paper (tests/golden), closed forms, brute force
on tiny inputs, library routines for special cases, and invariants.  Some
tests also plant a plausible mistake (a wrong bit order, a dropped term) in
a copy of an oracle step and show that the pin rejects it.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example_4x8x2.txt")


def _golden():
    rec = {"prefix": [], "segment": []}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        v = [int(x) for x in v]
        if k in ("prefix", "segment"):
            rec[k].append(v)
        else:
            rec[k] = v if len(v) > 1 else v[0]
    return rec


# ---------------------------------------------------------------------------
# encoding: the worked example of Sec. 3.1 / 3.2


def _decode_fn_oracle(dims):
    return lambda keys: oracle.decode(dims, np.stack([np.asarray(keys, np.uint64),
                                                      np.zeros(len(keys), np.uint64)], 1)).astype(np.int64)


def _decode_fn_from_positions(pos):
    """A decode built from an explicit bit map pos[n] = key bits of mode n
    (used to plant mistakes)."""
    def f(keys):
        out = np.zeros((len(keys), len(pos)), dtype=np.int64)
        for x, k in enumerate(keys):
            for n, ps in enumerate(pos):
                out[x, n] = sum(((int(k) >> p) & 1) << l for l, p in enumerate(ps))
        return out
    return f


def _worked_example_holds(decode, g):
    """True when a decode reproduces every statement of the worked example."""
    dims = g["dims"]
    B = int(math.log2(g["line_length"]))
    allk = np.arange(2 ** B)
    coords = decode(allk)
    # bijection of the 64-point line onto the 4 x 8 x 2 space
    if len({tuple(c) for c in coords}) != 2 ** B or any((coords[:, n] >= dims[n]).any() for n in range(3)):
        return False
    # prefixes encode boxes of the printed extents
    for lo, hi, *ext in g["prefix"]:
        c = coords[lo:hi + 1]
        for n in range(3):
            vals = np.unique(c[:, n])
            if len(vals) != ext[n] or vals.max() - vals.min() + 1 != ext[n]:
                return False
    # two equal-nnz segments with the printed endpoints and tight intervals:
    # some choice of the two middle nonzeros must reproduce them
    (a0, a1, *iv0), (b0, b1, *iv1) = g["segment"]

    def tight(keys, iv):
        c = decode(keys)
        return all(c[:, n].min() == iv[2 * n] and c[:, n].max() == iv[2 * n + 1] for n in range(3))
    ok0 = any(tight([a0, m, a1], iv0) for m in range(a0 + 1, a1))
    ok1 = any(tight([b0, m, b1], iv1) for m in range(b0 + 1, b1))
    return ok0 and ok1


def test_worked_example_line_length():
    g = _golden()
    nbits, pos, B = oracle.bit_map(g["dims"])
    assert 2 ** B == g["line_length"]
    assert list(nbits) == [2, 3, 1]


def test_worked_example_encoding():
    g = _golden()
    assert _worked_example_holds(_decode_fn_oracle(g["dims"]), g)


def test_worked_example_rejects_wrong_bit_orders():
    """Planted mistakes: longest mode first inside a level, a fixed i,j,k
    interleave, and plain row-major linearization all contradict the text."""
    g = _golden()
    longest_first = [[1, 4], [0, 3, 5], [2]]          # j, i, k inside a level
    fixed_ijk = [[0, 3], [1, 4, 5], [2]]               # i, j, k inside a level
    row_major = [[4, 5], [1, 2, 3], [0]]               # i*16 + j*2 + k
    for pos in (longest_first, fixed_ijk, row_major):
        assert not _worked_example_holds(_decode_fn_from_positions(pos), g)


def test_worked_example_partition_and_intervals():
    """Equal-nnz partitioning + tight intervals on a tensor consistent with
    the worked example reproduce the printed segments and intervals."""
    g = _golden()
    dims = g["dims"]
    dec = _decode_fn_oracle(dims)
    (a0, a1, *iv0), (b0, b1, *iv1) = g["segment"]
    found = 0
    for m0 in range(a0 + 1, a1):
        for m1 in range(b0 + 1, b1):
            keys = [a0, m0, a1, b0, m1, b1]
            coords = dec(keys)
            idx = [coords[:, n].astype(np.uint32) for n in range(3)]
            k = oracle.encode(dims, idx)
            perm = oracle.sort_perm(k)
            bounds = oracle.partition(6, 2)
            cs = oracle.decode(dims, k[perm])
            ivl = oracle.intervals(cs, bounds)
            if [list(ivl[0].ravel()), list(ivl[1].ravel())] == [iv0, iv1]:
                found += 1
                assert list(k[perm][:, 0][bounds[:-1]]) == [a0, b0]
                assert list(k[perm][:, 0][bounds[1:] - 1]) == [a1, b1]
    assert found > 0


def test_eq2_and_eq3_examples():
    g = _golden()
    wb, coo, alto_w, ratio = g["eq2"]
    assert oracle.compression_ratio(g["dims"], wb) == ratio == coo / alto_w
    nbits, _, B = oracle.bit_map(g["dims"])
    assert 2 ** oracle.sfc_bits(g["dims"]) // 2 ** B == g["sfc_ratio"]


def test_eq1_bits():
    # Eq. 1 with whole bits per mode; a length-1 mode needs none
    for dims, B in [((4, 8, 2), 6), ((4_000_000, 4_000_000, 30_000), 59),
                    ((12_000, 60_000, 5_000_000, 100), 60),
                    ((1 << 20,) * 3 + (1 << 16,) * 2, 92), ((1, 7, 1), 3), ((2 ** 32, 3), 34)]:
        assert oracle.bit_map(dims)[2] == B
        assert sum(oracle.bits_per_mode(dims)) == B


# ---------------------------------------------------------------------------
# encoding invariants (brute force on tiny grids)


@pytest.mark.parametrize("dims", [(4, 8, 2), (3, 5, 2), (1, 7, 3, 2), (2, 2, 2, 2, 2), (5, 1, 9), (16,)])
def test_encode_decode_bijection(dims):
    cells = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.int64)
    idx = [cells[:, n] for n in range(len(dims))]
    keys = oracle.encode(dims, idx)
    back = oracle.decode(dims, keys).astype(np.int64)
    assert (back == cells).all()
    B = oracle.bit_map(dims)[2]
    lin = keys[:, 0]
    assert len(np.unique(lin)) == len(cells)
    assert lin.max() < 2 ** B
    if all(d & (d - 1) == 0 for d in dims):   # powers of two: onto [0, 2^B)
        assert sorted(lin.tolist()) == list(range(2 ** B))


def test_level_structure_more_significant_bits_split_longer_modes():
    """Sec. 3.1: the most significant bit belongs to the longest mode and a
    key bit never belongs to a shorter mode than the bit above it inside a
    level; each mode's bits ascend with key position."""
    for dims in [(4_000_000, 4_000_000, 30_000), (12_000, 60_000, 5_000_000, 100), (7, 300, 2, 90)]:
        nbits, pos, B = oracle.bit_map(dims)
        owner = {}
        for n in range(len(dims)):
            ps = [pos[n][l] for l in range(nbits[n])]
            assert ps == sorted(ps)
            for p in ps:
                owner[p] = n
        assert sorted(owner) == list(range(B))
        assert dims[owner[B - 1]] == max(dims)


def test_128bit_keys():
    dims = (1 << 20,) * 3 + (1 << 16,) * 2
    rng = np.random.default_rng(0)
    idx = [rng.integers(0, d, 1000, dtype=np.int64) for d in dims]
    keys = oracle.encode(dims, idx)
    assert (keys[:, 1] > 0).any()
    back = oracle.decode(dims, keys).astype(np.int64)
    assert (back == np.stack(idx, 1)).all()


def test_encode_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.encode((4, 8), [np.array([0, 4]), np.array([0, 1])])


# ---------------------------------------------------------------------------
# ordering and partitioning


def test_sort_stable_matches_library_sort():
    rng = np.random.default_rng(1)
    keys = np.zeros((5000, 2), dtype=np.uint64)
    keys[:, 0] = rng.integers(0, 50, 5000).astype(np.uint64)       # many ties
    keys[:, 1] = rng.integers(0, 3, 5000).astype(np.uint64)
    perm = oracle.sort_perm(keys)
    ref = np.lexsort((np.arange(5000), keys[:, 0], keys[:, 1]))
    assert (perm == ref).all()
    assert (perm == np.lexsort((keys[:, 0], keys[:, 1]))).all()   # numpy lexsort is stable


@pytest.mark.parametrize("M,L", [(10, 3), (6, 2), (1000, 7), (5, 5), (7, 1), (0, 1)])
def test_partition_equal_nnz(M, L):
    b = oracle.partition(M, L)
    sizes = np.diff(b)
    assert b[0] == 0 and b[-1] == M and len(b) == L + 1
    assert (sizes >= 0).all() and sizes.max() - sizes.min() <= 1
    assert sizes.sum() == M


def test_intervals_tight_and_covering():
    rng = np.random.default_rng(2)
    dims = (50, 7, 300)
    idx = [rng.integers(0, d, 400) for d in dims]
    k = oracle.encode(dims, idx)
    perm = oracle.sort_perm(k)
    cs = oracle.decode(dims, k[perm]).astype(np.int64)
    b = oracle.partition(400, 9)
    ivl = oracle.intervals(cs, b).astype(np.int64)
    for l in range(9):
        seg = cs[b[l]:b[l + 1]]
        for n in range(3):
            assert (seg[:, n] >= ivl[l, n, 0]).all() and (seg[:, n] <= ivl[l, n, 1]).all()
            assert ivl[l, n, 0] in seg[:, n] and ivl[l, n, 1] in seg[:, n]


def test_flags_brute_force():
    rng = np.random.default_rng(3)
    dims = (40, 500, 6)
    idx = [rng.integers(0, d, 300) for d in dims]
    k = oracle.encode(dims, idx)
    perm = oracle.sort_perm(k)
    cs = oracle.decode(dims, k[perm]).astype(np.int64)
    b = oracle.partition(300, 11)
    for n in range(3):
        f = oracle.flags(cs, dims[n], n, b)
        segs_of_row = {}
        for l in range(11):
            for x in range(b[l], b[l + 1]):
                segs_of_row.setdefault(cs[x, n], set()).add(l)
        for x in range(300):
            assert f[x] == (len(segs_of_row[cs[x, n]]) == 1)


# ---------------------------------------------------------------------------
# MTTKRP


def _dense(dims, idx, vals):
    X = np.zeros(dims)
    np.add.at(X, tuple(np.asarray(i, dtype=np.int64) for i in idx), vals)
    return X


def _unfold(X, n):
    """Mode-n matricization (Sec. 2.2): mode-n fibers as columns; the column
    of (i_m)_{m != n} enumerates the remaining modes with the last fastest."""
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1)


def _khatri_rao(mats):
    """Column-wise Kronecker product [b_1 (x) c_1, ...] (Sec. 2.2)."""
    K = mats[0]
    for B in mats[1:]:
        K = np.einsum("ir,jr->ijr", K, B).reshape(-1, K.shape[1])
    return K


def _random_sparse(rng, dims, M, dup=False):
    idx = [rng.integers(0, d, M) for d in dims]
    if dup:
        for n in range(len(dims)):
            idx[n][M // 2:] = idx[n][:M - M // 2]
    return idx, rng.standard_normal(M)


@pytest.mark.parametrize("dims,M", [((5, 6, 7), 60), ((4, 3, 5, 2), 50), ((3, 4, 2, 3, 2), 40), ((9, 8), 30)])
def test_mttkrp_matches_dense_bruteforce(dims, M):
    rng = np.random.default_rng(4)
    idx, vals = _random_sparse(rng, dims, M, dup=True)
    R = 5
    U = [rng.standard_normal((d, R)) for d in dims]
    X = _dense(dims, idx, vals)
    for n in range(len(dims)):
        ref = _unfold(X, n) @ _khatri_rao([U[m] for m in range(len(dims)) if m != n])
        got = oracle.mttkrp(dims, idx, vals, U, n)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_mttkrp_bruteforce_rejects_dropped_term():
    """Planted mistake: leaving one factor out of the product is caught."""
    rng = np.random.default_rng(5)
    dims = (4, 5, 6)
    idx, vals = _random_sparse(rng, dims, 40)
    U = [rng.standard_normal((d, 3)) for d in dims]
    X = _dense(dims, idx, vals)
    ref = _unfold(X, 0) @ _khatri_rao([U[1], U[2]])
    wrong = [U[0], np.ones_like(U[1]), U[2]]     # drops U_1
    assert not np.allclose(oracle.mttkrp(dims, idx, vals, wrong, 0), ref)


def test_mttkrp_closed_form_dense_low_rank():
    """A fully dense X = [[U_1..U_N]] gives MTTKRP_n = U_n (Hadamard of U_m^T U_m)."""
    rng = np.random.default_rng(6)
    dims = (6, 5, 4, 3)
    R = 3
    U = [rng.standard_normal((d, R)) for d in dims]
    X = np.einsum("ir,jr,kr,lr->ijkl", *U)
    cells = np.array(list(itertools.product(*[range(d) for d in dims])))
    idx = [cells[:, n] for n in range(4)]
    vals = X[tuple(idx)]
    for n in range(4):
        H = np.ones((R, R))
        for m in range(4):
            if m != n:
                H *= U[m].T @ U[m]
        np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals, U, n), U[n] @ H, rtol=1e-11, atol=1e-11)


def test_mttkrp_order2_is_spmm():
    import scipy.sparse as sp
    rng = np.random.default_rng(7)
    dims = (30, 40)
    idx, vals = _random_sparse(rng, dims, 200, dup=True)
    A = sp.coo_matrix((vals, (idx[0], idx[1])), shape=dims).tocsr()
    B = rng.standard_normal((40, 4))
    C = rng.standard_normal((30, 4))
    np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals, [None, B], 0), A @ B, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals, [C, None], 1), A.T @ C, rtol=1e-12, atol=1e-12)
    x = rng.standard_normal((40, 1))     # R = 1: SpMV
    np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals, [None, x], 0), A @ x, rtol=1e-12, atol=1e-12)


def test_mttkrp_sampled_rows():
    rng = np.random.default_rng(8)
    dims = (50, 40, 30)
    idx, vals = _random_sparse(rng, dims, 500)
    U = [rng.standard_normal((d, 4)) for d in dims]
    full = oracle.mttkrp(dims, idx, vals, U, 2)
    rows = [0, 3, 17, 29]
    part = oracle.mttkrp(dims, idx, vals, U, 2, rows=rows)
    np.testing.assert_array_equal(part[rows], full[rows])
    mask = np.ones(30, bool)
    mask[rows] = False
    assert (part[mask] == 0).all()


def test_mttkrp_order_invariant():
    """ALTO reorders nonzeros: the MTTKRP of the ALTO-ordered tensor equals
    that of the input order (exactly up to rounding)."""
    rng = np.random.default_rng(9)
    dims = (20, 30, 10)
    idx, vals = _random_sparse(rng, dims, 300)
    k = oracle.encode(dims, idx)
    p = oracle.sort_perm(k)
    U = [rng.standard_normal((d, 6)) for d in dims]
    for n in range(3):
        np.testing.assert_allclose(oracle.mttkrp(dims, [i[p] for i in idx], vals[p], U, n),
                                   oracle.mttkrp(dims, idx, vals, U, n), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# conflict-resolution rule (Sec. 3.3) on the paper's own example


def test_conflict_rule_darpa_mode3_atomics():
    # darpa (Table 1): 22.5K x 22.5K x 23.8M, 28.4M nonzeros; Sec. 4.4.2 says
    # ALTO picks atomics for its mode-3 MTTKRP
    dims = (22_500, 22_500, 23_800_000)
    buf = oracle.use_buffered(dims, 28_400_000)
    assert buf == [True, True, False]
    # "more than" four operations: reuse exactly 4 stays with atomics
    assert oracle.use_buffered((10,), 40) == [False]
    assert oracle.use_buffered((10,), 41) == [True]


# ---------------------------------------------------------------------------
# CP-ALS (Kolda-Bader; Sec. 2.2)


def test_cpals_first_update_is_least_squares():
    """The mode-n update solves min ||X_(n) - U (KR of the others)^T||_F,
    checked against numpy's least-squares solver on the unfolded tensor."""
    rng = np.random.default_rng(10)
    dims = (6, 5, 4)
    idx, vals = _random_sparse(rng, dims, 70)
    R = 3
    U0 = [rng.standard_normal((d, R)) for d in dims]
    U, lam, fits, _ = oracle.cpals(dims, idx, vals, U0, 1)
    X = _dense(dims, idx, vals)
    K = _khatri_rao([U0[1], U0[2]])
    sol = np.linalg.lstsq(K, _unfold(X, 0).T, rcond=None)[0].T
    # after mode 0 of iteration 1 the factor is sol / its column 2-norms;
    # recompute it from a one-mode run
    Un = sol / np.sqrt((sol ** 2).sum(0))
    U1, _, _, _ = _cpals_modes(dims, idx, vals, U0, nmodes=1)
    np.testing.assert_allclose(U1[0], Un, rtol=1e-9, atol=1e-10)


def _cpals_modes(dims, idx, vals, U0, nmodes):
    """Oracle CP-ALS stopped after the first `nmodes` mode updates."""
    import scipy.linalg
    U = [u.copy() for u in U0]
    G = [u.T @ u for u in U]
    R = U[0].shape[1]
    for n in range(nmodes):
        Mn = oracle.mttkrp(dims, idx, vals, U, n)
        V = np.ones((R, R))
        for m in range(len(dims)):
            if m != n:
                V = V * G[m]
        Unew = scipy.linalg.cho_solve(scipy.linalg.cho_factor(V, lower=True), Mn.T).T
        lam = np.sqrt((Unew ** 2).sum(0))
        U[n] = Unew / lam
        G[n] = U[n].T @ U[n]
    return U, lam, None, None


def test_cpals_exact_recovery():
    rng = np.random.default_rng(11)
    dims = (7, 6, 5)
    R = 2
    T = [rng.standard_normal((d, R)) for d in dims]
    X = np.einsum("ir,jr,kr->ijk", *T)
    cells = np.array(list(itertools.product(*[range(d) for d in dims])))
    idx = [cells[:, n] for n in range(3)]
    vals = X[tuple(idx)]
    U0 = [t + 0.05 * rng.standard_normal(t.shape) for t in T]
    U, lam, fits, _ = oracle.cpals(dims, idx, vals, U0, 30)
    assert fits[-1] > 1 - 1e-6
    model = np.einsum("r,ir,jr,kr->ijk", lam, *U)
    np.testing.assert_allclose(model, X, rtol=1e-5, atol=1e-5)


def test_cpals_fit_matches_explicit_residual_and_is_monotone():
    rng = np.random.default_rng(12)
    dims = (8, 7, 6)
    idx, vals = _random_sparse(rng, dims, 150)
    R = 3
    U0 = [rng.random((d, R)) for d in dims]
    U, lam, fits, _ = oracle.cpals(dims, idx, vals, U0, 12)
    X = _dense(dims, idx, vals)
    model = np.einsum("r,ir,jr,kr->ijk", lam, *U)
    explicit = 1 - np.linalg.norm(X - model) / np.linalg.norm(X)
    assert abs(fits[-1] - explicit) < 1e-9
    assert all(b >= a - 1e-9 for a, b in zip(fits, fits[1:]))


def test_threaded_mttkrp_is_bit_identical():
    """The host-thread MTTKRP used for the multi-core CPU baseline performs the
    same additions per output element in the same order as the serial oracle."""
    import synth
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=50_000)
    dims, idx, vals = synth.tensor(cfg)
    rng = np.random.default_rng(5)
    U = [rng.standard_normal((d, 8)) for d in dims]
    for n in range(3):
        a = oracle.mttkrp(dims, idx, vals, U, n)
        b, used = oracle.mttkrp_threads(dims, idx, vals, U, n, 4)
        assert used >= 1
        assert np.array_equal(a, b)


def test_sampled_mttkrp_equals_full_rows():
    """Sampled-row MTTKRP (nonzeros filtered by output row, input rows
    relabeled) gives exactly the rows of the full oracle MTTKRP."""
    import synth
    cfg = synth.scaled("zipf3d-4Mx4Mx30k", nnz=40_000)
    cfg["dims"] = (30_000, 20_000, 3000)
    dims, idx, vals = synth.tensor(cfg)
    rng = np.random.default_rng(9)
    U = [rng.standard_normal((d, 8)) for d in dims]
    for n in range(3):
        full = oracle.mttkrp(dims, idx, vals, U, n)
        rows = np.sort(rng.choice(dims[n], size=500, replace=False))
        got = oracle.mttkrp_sampled(dims, idx, vals, lambda m, ids: U[m][ids], n, rows)
        assert np.array_equal(got, full[rows])


# ---------------------------------------------------------------------------
# transposition (Sec. 5: sorting the nonzeros by their coordinates in the new
# mode order)


def _transpose_bruteforce(dims, idx, modes):
    """No sort: walk the chosen modes' coordinate tuples in lexicographic
    order (itertools.product over their ranges) and list the nonzeros that
    hold each tuple, those by ascending ALTO key, then input position."""
    keys = oracle.encode(dims, idx)
    by = {}
    for x in range(len(idx[0])):
        by.setdefault(tuple(int(idx[m][x]) for m in modes), []).append(x)
    out = []
    for t in itertools.product(*[range(dims[m]) for m in modes]):
        out += sorted(by.get(t, []), key=lambda x: (int(keys[x, 1]), int(keys[x, 0]), x))
    return np.array(out, dtype=np.int64)


def _random_coo(dims, M, seed):
    """Coordinates drawn with replacement (so duplicates occur)."""
    rng = np.random.default_rng(seed)
    return [rng.integers(0, d, M).astype(np.uint32) for d in dims]


@pytest.mark.parametrize("dims,M", [((4, 8, 2), 40), ((5, 3, 7), 120), ((3, 4, 2, 5), 90), ((9,), 30)])
def test_transpose_matches_bruteforce(dims, M):
    idx = _random_coo(dims, M, sum(dims))
    N = len(dims)
    sels = [list(p) for p in itertools.permutations(range(N))]
    sels += [[m] for m in range(N)] + [list(p) for p in itertools.permutations(range(N), 2)][:6]
    for modes in sels:
        order, src = oracle.transpose(dims, idx, modes)
        assert np.array_equal(src, _transpose_bruteforce(dims, idx, modes)), modes
        # order indexes ALTO order: the ALTO-ordered input positions under it
        alto = oracle.sort_perm(oracle.encode(dims, idx))
        assert np.array_equal(alto[order], src)


def test_transpose_rejects_most_significant_first():
    """Planted mistake: applying the stable per-mode sorts most significant
    mode first (instead of last) breaks the lexicographic order."""
    dims = (5, 3, 7)
    idx = _random_coo(dims, 120, 15)
    modes = [2, 0, 1]
    alto = oracle.sort_perm(oracle.encode(dims, idx))
    coords = np.stack([np.asarray(a, np.int64)[alto] for a in idx], 1)
    order = np.arange(len(alto))
    for m in modes:
        order = order[np.argsort(coords[order, m], kind="stable")]
    assert not np.array_equal(alto[order], _transpose_bruteforce(dims, idx, modes))


def test_transpose_full_order_of_distinct_coordinates_is_unique():
    """With distinct coordinates and every mode chosen, the result is the
    unique strictly increasing lexicographic sequence, whatever the input
    order."""
    rng = np.random.default_rng(3)
    dims = (50, 40, 30)
    flat = rng.choice(50 * 40 * 30, size=5000, replace=False)
    idx = [(flat // (40 * 30)).astype(np.uint32), ((flat // 30) % 40).astype(np.uint32),
           (flat % 30).astype(np.uint32)]
    for modes in ([0, 1, 2], [2, 0, 1], [1, 2, 0]):
        _, src = oracle.transpose(dims, idx, modes)
        c = np.stack([np.asarray(idx[m], np.int64)[src] for m in modes], 1)
        lin = (c[:, 0] * dims[modes[1]] + c[:, 1]) * dims[modes[2]] + c[:, 2]
        assert (np.diff(lin) > 0).all()
        shuffled = rng.permutation(len(flat))
        _, src2 = oracle.transpose(dims, [a[shuffled] for a in idx], modes)
        assert np.array_equal(shuffled[src2], src)
