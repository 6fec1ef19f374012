/*
 * Plain FP64 CPU oracle for the ALTO hot path (Helal et al., "ALTO: Adaptive
 * Linearized Storage of Sparse Tensors", ICS '21).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Everything here is written to be checked against the paper by eye:
 * no blocking, no fusion, no reordering beyond what the paper states.
 *
 *   orc_bit_map      Sec. 3.1 (Fig. 2 text): bits per mode, level-by-level
 *                    assignment starting at the LSB, shortest mode first
 *                    inside a level; Eq. 1 for the bit count.
 *   orc_encode       Sec. 3.1: linearization, one key bit at a time.
 *   orc_decode       Sec. 3.1 / Alg. 1 EXTRACT: de-linearization, one bit at
 *                    a time.
 *   orc_sort_perm    Sec. 3.1 ordering stage: ascending key, ties kept in
 *                    input order.
 *   orc_partition    Sec. 3.2: L line segments with equal nonzero counts.
 *   orc_intervals    Sec. 3.2: closed per-mode intervals T_{l,n} of each
 *                    segment (tight min/max over the segment's elements).
 *   orc_flags        Sec. 3.3 last paragraph: boundary/internal element flag
 *                    along a mode (internal = its row is touched by exactly
 *                    one segment).
 *   orc_mttkrp       Sec. 2.2 definition / Alg. 1 in COO form: direct
 *                    summation out[i_n][r] += v * prod_{m!=n} U_m[i_m][r].
 *   orc_mttkrp_threads  the same sums on several host threads: thread t
 *                    owns the output rows i_n with i_n mod T == t and adds
 *                    their nonzeros in input order, so every output row is
 *                    the same sequence of FP64 additions as in orc_mttkrp
 *                    (bit-identical results); only used to time the oracle
 *                    on all host cores.
 *
 * Keys are always held as two 64-bit words per nonzero (lo, hi), whatever
 * the word width the product path picks.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 16
#define ORC_MAXB 128

/* Number of bits that mode length I needs: the smallest b with 2^b >= I
 * (Eq. 1 prints log2 I_n; a length of 1 needs no bit). */
static int bits_for_length(uint64_t I)
{
    int b = 0;
    while (b < 64 && ((uint64_t)1 << b) < I)
        b++;
    return b;
}

/*
 * Bit map of the ALTO index (Sec. 3.1): walk the levels l = 0, 1, ... from
 * the least significant end; inside one level visit the modes in increasing
 * order of their length (ties: lower mode index first); every mode that
 * still has a bit at this level takes the next free key position.
 * pos[n * ORC_MAXB + l] = key bit holding bit l of the mode-n index.
 * Returns the total number of bits B (Eq. 1), or -1 on bad input.
 */
int orc_bit_map(int N, const uint64_t *dims, int *nbits, int *pos)
{
    int order[ORC_MAXN];
    int n, l, a, maxb = 0, next = 0;
    if (N < 1 || N > ORC_MAXN)
        return -1;
    for (n = 0; n < N; n++) {
        if (dims[n] < 1)
            return -1;
        nbits[n] = bits_for_length(dims[n]);
        if (nbits[n] > maxb)
            maxb = nbits[n];
        order[n] = n;
        for (l = 0; l < ORC_MAXB; l++)
            pos[n * ORC_MAXB + l] = -1;
    }
    /* insertion sort of the modes by (length, index) */
    for (a = 1; a < N; a++) {
        int m = order[a], b = a - 1;
        while (b >= 0 && (dims[order[b]] > dims[m] ||
                          (dims[order[b]] == dims[m] && order[b] > m))) {
            order[b + 1] = order[b];
            b--;
        }
        order[b + 1] = m;
    }
    for (l = 0; l < maxb; l++)
        for (a = 0; a < N; a++) {
            n = order[a];
            if (l < nbits[n])
                pos[n * ORC_MAXB + l] = next++;
        }
    return next;
}

static void set_bit(uint64_t *key2, int p)
{
    key2[p >> 6] |= (uint64_t)1 << (p & 63);
}

static int get_bit(const uint64_t *key2, int p)
{
    return (int)((key2[p >> 6] >> (p & 63)) & 1u);
}

static uint64_t read_index(const void *arr, int idx_bytes, int64_t x)
{
    if (idx_bytes == 4)
        return ((const uint32_t *)arr)[x];
    return (uint64_t)((const int64_t *)arr)[x];
}

/*
 * Linearization (Sec. 3.1): for every nonzero x and every mode n, copy bit l
 * of i_n to key position pos(n, l).  idx[n] points to M indices of mode n
 * (idx_bytes = 4 or 8).  keys receives 2*M words (lo, hi) per nonzero.
 * Returns 0, or the 1-based mode of the first out-of-range index as a
 * negative number.
 */
int orc_encode(int N, const uint64_t *dims, int64_t M, const void *const *idx,
               int idx_bytes, uint64_t *keys)
{
    int nbits[ORC_MAXN];
    int *pos = (int *)malloc(sizeof(int) * ORC_MAXN * ORC_MAXB);
    int64_t x;
    int n, l;
    if (!pos || orc_bit_map(N, dims, nbits, pos) < 0) {
        free(pos);
        return -1000;
    }
    for (x = 0; x < M; x++) {
        uint64_t *k = keys + 2 * x;
        k[0] = 0;
        k[1] = 0;
        for (n = 0; n < N; n++) {
            uint64_t i = read_index(idx[n], idx_bytes, x);
            if (i >= dims[n]) {
                free(pos);
                return -(n + 1);
            }
            for (l = 0; l < nbits[n]; l++)
                if ((i >> l) & 1u)
                    set_bit(k, pos[n * ORC_MAXB + l]);
        }
    }
    free(pos);
    return 0;
}

/* De-linearization (EXTRACT of Alg. 1): the inverse bit walk.  out is M x N
 * row-major (out[x * N + n] = i_n of nonzero x). */
int orc_decode(int N, const uint64_t *dims, int64_t M, const uint64_t *keys,
               uint64_t *out)
{
    int nbits[ORC_MAXN];
    int *pos = (int *)malloc(sizeof(int) * ORC_MAXN * ORC_MAXB);
    int64_t x;
    int n, l;
    if (!pos || orc_bit_map(N, dims, nbits, pos) < 0) {
        free(pos);
        return -1;
    }
    for (x = 0; x < M; x++)
        for (n = 0; n < N; n++) {
            uint64_t i = 0;
            for (l = 0; l < nbits[n]; l++)
                if (get_bit(keys + 2 * x, pos[n * ORC_MAXB + l]))
                    i |= (uint64_t)1 << l;
            out[x * N + n] = i;
        }
    free(pos);
    return 0;
}

/* Ordering stage (Sec. 3.1): sort positions by (hi, lo) key, ties by the
 * original position so that equal keys keep their input order. */
static const uint64_t *g_sort_keys;

static int cmp_key_then_index(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    const uint64_t *ka = g_sort_keys + 2 * a, *kb = g_sort_keys + 2 * b;
    if (ka[1] != kb[1])
        return ka[1] < kb[1] ? -1 : 1;
    if (ka[0] != kb[0])
        return ka[0] < kb[0] ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* perm[i] = input position of the i-th nonzero in ALTO order. */
int orc_sort_perm(int64_t M, const uint64_t *keys, int64_t *perm)
{
    int64_t x;
    for (x = 0; x < M; x++)
        perm[x] = x;
    g_sort_keys = keys;
    qsort(perm, (size_t)M, sizeof(int64_t), cmp_key_then_index);
    g_sort_keys = NULL;
    return 0;
}

/* Equal-nnz line segments (Sec. 3.2): bounds[l] = floor(l * M / L),
 * l = 0..L; segment l holds the ordered positions [bounds[l], bounds[l+1]). */
int orc_partition(int64_t M, int64_t L, int64_t *bounds)
{
    int64_t l;
    if (L < 1)
        return -1;
    for (l = 0; l <= L; l++) {
        /* floor(l*M/L) without overflow for the sizes used here */
        __int128 t = (__int128)l * (__int128)M;
        bounds[l] = (int64_t)(t / L);
    }
    return 0;
}

/*
 * Mode intervals of every segment (Sec. 3.2): T_{l,n} = [min, max] of the
 * mode-n index over the segment's elements.  coords is the decoded M x N
 * array in ALTO order.  ivl has L x N x 2 entries (start, end); an empty
 * segment gets (1, 0).
 */
int orc_intervals(int N, int64_t M, const uint64_t *coords, int64_t L,
                  const int64_t *bounds, uint64_t *ivl)
{
    int64_t l, x;
    int n;
    (void)M;
    for (l = 0; l < L; l++)
        for (n = 0; n < N; n++) {
            uint64_t lo = 1, hi = 0;
            int first = 1;
            for (x = bounds[l]; x < bounds[l + 1]; x++) {
                uint64_t i = coords[x * N + n];
                if (first || i < lo)
                    lo = i;
                if (first || i > hi)
                    hi = i;
                first = 0;
            }
            ivl[(l * N + n) * 2 + 0] = lo;
            ivl[(l * N + n) * 2 + 1] = hi;
        }
    return 0;
}

/*
 * Helper flags (Sec. 3.3, last paragraph) along mode n: flag[x] = 1 when the
 * mode-n row of element x is touched by exactly one segment (internal /
 * exclusive element), 0 when several segments touch it (boundary element).
 * coords in ALTO order; owner/count scratch are sized I_n.
 */
int orc_flags(int N, uint64_t In, int n, int64_t M, const uint64_t *coords,
              int64_t L, const int64_t *bounds, uint8_t *flag)
{
    int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * (size_t)In);
    int64_t *nseg = (int64_t *)malloc(sizeof(int64_t) * (size_t)In);
    int64_t l, x;
    uint64_t r;
    if (!owner || !nseg) {
        free(owner);
        free(nseg);
        return -1;
    }
    for (r = 0; r < In; r++) {
        owner[r] = -1;
        nseg[r] = 0;
    }
    for (l = 0; l < L; l++)
        for (x = bounds[l]; x < bounds[l + 1]; x++) {
            uint64_t i = coords[x * N + n];
            if (owner[i] != l) {       /* first time segment l meets row i */
                owner[i] = l;          /* segments are visited in order, so */
                nseg[i] += 1;          /* a row is counted once per segment */
            }
        }
    for (x = 0; x < M; x++)
        flag[x] = (uint8_t)(nseg[coords[x * N + n]] == 1);
    free(owner);
    free(nseg);
    return 0;
}

/*
 * Mode-n MTTKRP by its definition (Sec. 2.2; Alg. 1 in COO form):
 *   out[i_n][r] = sum over nonzeros x of v_x * prod_{m != n} U_m[i_m][r]
 * summed in input order, FP64.  factors[m] is I_m x R row-major (ld = R);
 * factors[n] is not read.  out (I_n x R) is overwritten.  When rowmask is
 * not NULL only rows with rowmask[i_n] != 0 are accumulated (the others are
 * left at zero).
 */
int orc_mttkrp(int N, const uint64_t *dims, int64_t M, const void *const *idx,
               int idx_bytes, const double *vals, const double *const *factors,
               int R, int n, const uint8_t *rowmask, double *out)
{
    int64_t x;
    int m, r;
    uint64_t i[ORC_MAXN];
    memset(out, 0, sizeof(double) * (size_t)dims[n] * (size_t)R);
    for (x = 0; x < M; x++) {
        for (m = 0; m < N; m++)
            i[m] = read_index(idx[m], idx_bytes, x);
        if (rowmask && !rowmask[i[n]])
            continue;
        for (r = 0; r < R; r++) {
            double t = vals[x];
            for (m = 0; m < N; m++)
                if (m != n)
                    t *= factors[m][i[m] * (uint64_t)R + r];
            out[i[n] * (uint64_t)R + r] += t;
        }
    }
    return 0;
}

/*
 * orc_mttkrp on `threads` host threads (OpenMP): every thread reads all
 * nonzeros and accumulates those whose output row it owns (i_n mod T), in
 * input order.  Each output element receives the same additions in the same
 * order as in orc_mttkrp.  Returns the number of threads used.
 */
int orc_mttkrp_threads(int N, const uint64_t *dims, int64_t M, const void *const *idx,
                       int idx_bytes, const double *vals, const double *const *factors,
                       int R, int n, double *out, int threads)
{
    int used = 1;
    if (threads < 1)
        threads = 1;
    memset(out, 0, sizeof(double) * (size_t)dims[n] * (size_t)R);
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
    {
        const uint64_t T = (uint64_t)omp_get_num_threads();
        const uint64_t me = (uint64_t)omp_get_thread_num();
        int64_t x;
        int m, r;
        uint64_t i[ORC_MAXN];
#pragma omp single
        used = (int)T;
        for (x = 0; x < M; x++) {
            const uint64_t row = read_index(idx[n], idx_bytes, x);
            if (row % T != me)
                continue;
            for (m = 0; m < N; m++)
                i[m] = read_index(idx[m], idx_bytes, x);
            for (r = 0; r < R; r++) {
                double t = vals[x];
                for (m = 0; m < N; m++)
                    if (m != n)
                        t *= factors[m][i[m] * (uint64_t)R + r];
                out[row * (uint64_t)R + r] += t;
            }
        }
    }
#else
    (void)threads;
    orc_mttkrp(N, dims, M, idx, idx_bytes, vals, factors, R, n, NULL, out);
#endif
    return used;
}
