/*
 * alto.h -- C ABI of libalto, a GB300 (sm_103a) implementation of the ALTO
 * sparse tensor format and of the MTTKRP / CP-ALS computations over it
 * (Helal et al., "ALTO: Adaptive Linearized Storage of Sparse Tensors",
 * ICS '21).
 *
 * Conventions shared by every entry point:
 *   - Plain pointers and sizes only.  `stream` is a cudaStream_t passed as
 *     void* (NULL = the legacy default stream).  Work is enqueued on that
 *     stream and runs asynchronously unless the entry point says it syncs.
 *   - Every function returns an alto_status; on failure alto_last_error()
 *     returns a message for the calling thread.  No C++ exception crosses
 *     the ABI.
 *   - Mode numbers are 0-based (the paper counts modes from 1).
 *   - Factor matrices are row-major I_m x R with leading dimension R.
 *   - Device-side errors (an index >= I_n, a bounded wait that ran out) are
 *     recorded in a status word owned by the tensor and reported by the next
 *     call that synchronises (alto_create, alto_cpals, alto_check).
 *   - The library owns every buffer it allocates and frees it in
 *     alto_destroy; caller buffers are only read or written, never freed.
 */
#ifndef ALTO_H
#define ALTO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct alto_tensor_s *alto_t;
typedef struct alto_batch_s *alto_batch_t;

typedef enum {
    ALTO_OK = 0,
    ALTO_EINVAL = 1,    /* bad argument (null pointer, bad mode, bad dtype) */
    ALTO_ENOMEM = 2,    /* an allocation failed */
    ALTO_ECUDA = 3,     /* a CUDA runtime call failed */
    ALTO_ETIMEOUT = 4,  /* a bounded device wait ran out */
    ALTO_EOVERFLOW = 5, /* sum of index bits above 128 */
    ALTO_ENOTSPD = 6,   /* Cholesky factorisation of the Gram product failed */
    ALTO_ERANGE = 7     /* an input index is >= its mode length */
} alto_status;

typedef enum {
    ALTO_F64 = 0,
    ALTO_F32 = 1,
    ALTO_BF16 = 2
} alto_dtype;

/* Output-accumulation variants of MTTKRP (Alg. 2 and Sec. 3.3). */
typedef enum {
    ALTO_VAR_AUTO = 0,    /* the library's choice (Sec. 3.3 reuse rule:
                             reuse <= 4 -> ATOMIC, else WARPAGG) */
    ALTO_VAR_ATOMIC = 1,  /* direct atomic update per nonzero (Alg. 2, ATOMIC) */
    ALTO_VAR_WARPAGG = 2, /* warp-level pre-aggregation of equal output rows,
                             then atomics */
    ALTO_VAR_SMEM = 3,    /* per-segment Temp in shared memory sized by the
                             segment's output interval (Alg. 2, Temp_l), then
                             one atomic flush per touched row */
    ALTO_VAR_TEMP = 4     /* per-segment Temp in device memory plus the
                             pull-based reduction of Alg. 2 */,
    ALTO_VAR_GENERIC = 5  /* the kernel for any order and rank (no rank or
                             order specialisation; one warp per segment,
                             scalar atomics): the baseline of the
                             rank-specialisation comparison (Sec. 4.5) */
} alto_variant;

/* Engine of the Gram matrices U^T U of CP-ALS and alto_gram. */
typedef enum {
    ALTO_GRAM_AUTO = 0,          /* tensor cores for BF16 factors with R in
                                    {8, 16, 32, 64}, CUDA cores otherwise */
    ALTO_GRAM_CUDA_CORES = 1,    /* FP32 (FP64 for FP64 factors) partial sums
                                    on the CUDA cores, FP64 across blocks */
    ALTO_GRAM_TENSOR_CORES = 2   /* tcgen05 kind::f16 MMA: exact BF16
                                    products, FP32 sums per thread block in
                                    tensor memory, FP64 across blocks (BF16
                                    factors and R in {8, 16, 32, 64} only) */
} alto_gram_engine;

#define ALTO_MAX_MODES 8

/*
 * Creation options.  Zero-initialise, or call alto_options_init.
 *   key_bits : 0 = smallest native word that holds the index (64 or 128,
 *              Sec. 4.2.3) for generation and export, with the stored MTTKRP
 *              keys packed into the fewest 32-bit words (alto_get_key_bytes);
 *              64 or 128 forces that full width everywhere (64 fails with
 *              ALTO_EOVERFLOW when the index needs more bits).
 *   nparts   : number L of equal-nnz line segments (Sec. 3.2); 0 = auto:
 *              segments of 2048 nonzeros, halved down to 256 while the
 *              tensor gives fewer than two thread-block units (8 segments
 *              each) per SM.
 *   variant  : per-mode MTTKRP variant (alto_variant); 0 = auto.
 *   use_flags: 1 = store boundary/internal helper flags in the unused key
 *              bits for modes whose fiber reuse is at most 4 (Sec. 3.3).
 *   alloc/free/ctx: optional device allocator; when alloc is NULL the
 *              library uses cudaMalloc / cudaFree.  alloc returns NULL on
 *              failure, which the library reports as ALTO_ENOMEM.
 */
typedef struct {
    int key_bits;
    int64_t nparts;
    int variant[ALTO_MAX_MODES];
    int use_flags;
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} alto_options;

/* Fill *opt with the defaults (all automatic, flags on, cudaMalloc). */
alto_status alto_options_init(alto_options *opt);

/*
 * alto_create -- build the ALTO tensor from a COO tensor (Sec. 3.1-3.2).
 *
 * Linearization (bit-level gather of every mode index into one key, bits
 * assigned level by level from the LSB, shorter modes first inside a level;
 * Sec. 3.1, Eq. 1), ordering (stable ascending sort of the keys), value
 * permutation, equal-nnz partitioning into L line segments with their
 * per-mode intervals T_l (Sec. 3.2), per-mode distinct-row counts and fiber
 * reuse, and the helper flags (Sec. 3.3).
 *
 *   out      : receives the handle.
 *   nmodes   : N, 1 <= N <= ALTO_MAX_MODES.
 *   dims     : host array of N mode lengths, each in [1, 2^32].
 *   nnz      : M >= 0 nonzeros (duplicates are kept as separate nonzeros).
 *   idx      : host array of N pointers; idx[n] points to M mode-n indices
 *              (0-based) of width idx_bytes (4: uint32, 8: int64).  Each
 *              pointer may be device or host memory (detected); host data is
 *              copied to the device first.
 *   vals     : M values of type vdtype (ALTO_F64, ALTO_F32 or ALTO_BF16),
 *              device or host memory.  BF16 values are stored as BF16 (2 bytes
 *              in the streamed format) and widened exactly to FP32 inside
 *              the MTTKRP kernels; they go with FP32 or BF16 factors.
 *   opt      : options, or NULL for the defaults.
 * The inputs are read only and may be freed once the call returns.  The
 * call synchronises `stream` at its end and returns ALTO_ERANGE when an
 * index is out of range.
 */
alto_status alto_create(alto_t *out, int nmodes, const uint64_t *dims,
                        int64_t nnz, const void *const *idx, int idx_bytes,
                        const void *vals, alto_dtype vdtype,
                        const alto_options *opt, void *stream);

/*
 * alto_mttkrp -- mode-`mode` MTTKRP over the ALTO tensor (Sec. 2.2,
 * Alg. 1-2): out[i_n][r] = sum_x v_x * prod_{m != n} U_m[i_m][r].
 *
 *   factors : host array of N device pointers, factors[m] an I_m x rank
 *             matrix of fdtype; factors[mode] is not read (may be NULL).
 *   fdtype  : ALTO_F64 (values must be F64), ALTO_F32 or ALTO_BF16 (values
 *             must be F32 or BF16; accumulation in FP32).
 *   out     : device I_mode x rank matrix, FP64 when fdtype is ALTO_F64 and
 *             FP32 otherwise; overwritten (the zero initialisation that
 *             Alg. 2 leaves implicit is done here).
 * Asynchronous on `stream`.  Scratch memory (Temp buffers of the
 * ALTO_VAR_TEMP variant) is allocated on first use and kept in the handle.
 */
alto_status alto_mttkrp(alto_t t, int mode, const void *const *factors,
                        int rank, alto_dtype fdtype, void *out, void *stream);

/*
 * alto_cpals -- `iters` iterations of CP-ALS (Sec. 2.2) with ALTO MTTKRP.
 * Per mode n: M_n = MTTKRP_n; V = Hadamard product of U_m^T U_m over
 * m != n (FP64); U_n = M_n V^{-1} through a Cholesky factorisation of V in
 * FP64 (for FP32/BF16 factors the FP64 inverse is rounded to FP32 and
 * applied with FP32 arithmetic); columns normalised by their 2-norm in the
 * first iteration and by max(1, max |.|) afterwards, the norms going to
 * lambda; U_n^T U_n recomputed (FP64 across thread blocks; on the tensor
 * cores for BF16 factors, see alto_gram_engine).  The fit after each iteration is
 * 1 - ||X - [[lambda; U]]|| / ||X||.
 *
 *   factors : host array of N device pointers to I_m x rank matrices of
 *             fdtype: the initial factors on entry, the result on return.
 *   lambda  : device array of rank doubles (output).
 *   fit     : host array of `iters` doubles (output), or NULL.
 * Synchronises `stream` at its end when fit is not NULL.
 */
alto_status alto_cpals(alto_t t, int rank, int iters, void *const *factors,
                       alto_dtype fdtype, double *lambda, double *fit,
                       void *stream);

/*
 * alto_get_layout -- the index layout (Sec. 3.1).  Any output may be NULL.
 *   nmodes        : N.
 *   bits_per_mode : N entries, ceil(log2 I_n).
 *   masks         : N x 2 words (lo, hi): key bits that hold mode n.
 *   key_words     : 1 (64-bit keys) or 2 (128-bit keys).
 *   flag_bit      : N entries, the key bit of mode n's boundary/internal
 *                   helper flag (Sec. 3.3, modes with reuse <= 4) or -1.
 *   hot_bit       : N entries, the key bit flagging elements whose mode-n row
 *                   is one of the mode's hot rows (modes with reuse > 4), or
 *                   -1.  Both kinds of flag live in the unused key bits above
 *                   the index and never widen the key.
 */
alto_status alto_get_layout(alto_t t, int *nmodes, int *bits_per_mode,
                            uint64_t *masks, int *key_words, int *flag_bit,
                            int *hot_bit);

/*
 * alto_get_hot_rows -- the hot rows of one mode, hottest first: the rows
 * with the largest counts when every 16th nonzero in ALTO order is counted,
 * at most 1024 of them (all rows whose sampled count reaches the smallest
 * power of two that keeps the list within that bound, counting only rows
 * sampled at least twice).  MTTKRP keeps the leading ones in a per-block
 * shared-memory copy.  rows: host array of at least 1024 entries, or NULL;
 * count: number of hot rows.
 */
alto_status alto_get_hot_rows(alto_t t, int mode, uint32_t *rows, int *count);

/*
 * alto_get_stats -- plan statistics (Sec. 3.2-3.3).  Any output may be NULL.
 *   nnz, nparts : M and L.
 *   distinct    : N entries, number of distinct mode-n indices D_n.
 *   reuse       : N entries, fiber reuse M / I_n.
 *   variant     : N entries, the MTTKRP variant the plan uses per mode.
 *   max_interval: N entries, the widest segment interval per mode.
 */
alto_status alto_get_stats(alto_t t, int64_t *nnz, int64_t *nparts,
                           uint64_t *distinct, double *reuse, int *variant,
                           uint64_t *max_interval);

/*
 * alto_export -- copy the format to HOST buffers (synchronises).  Any
 * output may be NULL.
 *   keys      : M x key_words uint64 (lo word first), ALTO order, with the
 *               flag bits included.
 *   perm      : M uint32, input position of each nonzero in ALTO order.
 *   vals      : M values of the tensor's value dtype, ALTO order.
 *   bounds    : L+1 segment boundaries.
 *   intervals : L x N x 2 uint32, [start, end] of every segment and mode.
 */
alto_status alto_export(alto_t t, uint64_t *keys, uint32_t *perm, void *vals,
                        int64_t *bounds, uint32_t *intervals);

/*
 * alto_gram -- G = U^T U (Sec. 2.2: the Gram matrices whose Hadamard product
 * is the CP-ALS system matrix V) for a device factor U (I x R row-major, R <=
 * 64, dtype F64 / F32 / BF16) into the device R x R FP64 matrix G
 * (overwritten).  `engine` is an alto_gram_engine; ALTO_GRAM_TENSOR_CORES
 * with FP32/FP64 factors or another R is ALTO_EINVAL.  Runs on `stream` and
 * synchronises it; ALTO_ETIMEOUT if a bounded device wait of the tensor-core
 * kernel ran out (G is then incomplete).  All alto_gram calls share one
 * device status word: calls that overlap on the GPU may report each other's
 * timeout.
 */
alto_status alto_gram(const void *U, int64_t I, int R, alto_dtype dtype,
                      int engine, double *G, void *stream);

/* alto_set_gram_engine -- the engine alto_cpals uses for this tensor's Gram
 * matrices (ALTO_GRAM_AUTO by default).  Errors: ALTO_EINVAL for a NULL
 * handle or an unknown engine. */
alto_status alto_set_gram_engine(alto_t t, int engine);

/*
 * alto_transpose -- sparse tensor transposition (Sec. 5, sparse tensor
 * operations): the nonzeros in the lexicographic order of the coordinates of
 * modes[0], modes[1], ..., modes[nsel-1] (modes[0] most significant).  The
 * sort key is cut out of the stored linearized index and sorted by a stable
 * LSD radix sort over the chosen modes' index bits only (a partial radix
 * sort: sum of b_m over the chosen modes, not all B bits).  Nonzeros that tie
 * on the chosen modes keep ALTO order; with nsel = N only duplicate
 * coordinates tie, and they keep input order.
 *   nsel, modes : 1 <= nsel <= N distinct modes (host array).
 *   order       : device, M uint32 or NULL: ALTO position of the y-th nonzero
 *                 of the result.
 *   src         : device, M uint32 or NULL: its input position (the index of
 *                 the nonzero in the arrays given to alto_create).
 *   idx         : host array of N device pointers, or NULL: coordinates of the
 *                 result, M entries of idx_bytes (4: uint32, 8: int64) each;
 *                 output mode j is modes[j] for j < nsel, the remaining modes
 *                 follow in ascending order.
 *   vals        : device, M values of the stored value dtype, or NULL.
 * Runs on `stream` and synchronises it before returning (the sort scratch,
 * 2 x M x (8 or 16) + 2 x M x 4 bytes, is allocated through the tensor's
 * allocator and freed).  Errors: ALTO_EINVAL (NULL handle, nsel outside
 * [1, N], a repeated or out-of-range mode, idx_bytes not 4 or 8, a NULL
 * coordinate pointer), ALTO_ENOMEM, ALTO_ECUDA.  An empty tensor writes
 * nothing.
 */
alto_status alto_transpose(alto_t t, int nsel, const int *modes,
                           uint32_t *order, uint32_t *src, void *const *idx,
                           int idx_bytes, void *vals, void *stream);

/*
 * alto_get_mode_stats -- statistics of one mode, for variant selection.
 * out[0..n) (n <= 8 used): 0 length I_n, 1 distinct rows D_n, 2 reuse M/I_n,
 * 3 widest segment interval, 4 hot rows, 5 share of the sampled nonzeros
 * that fall in the hot rows, 6 median and 7 90th-percentile width of the
 * thread-block units' intervals (8 consecutive segments).
 */
alto_status alto_get_mode_stats(alto_t t, int mode, double *out, int n);

/* alto_get_unit_fit -- fraction of thread-block units whose mode-`mode`
 * interval has at most `rows` rows (how often a shared Temp of that many rows
 * holds a unit's output). */
alto_status alto_get_unit_fit(alto_t t, int mode, uint64_t rows, double *frac);

/*
 * Kernels of the variant-predictor MLP (row-major FP32, device pointers,
 * asynchronous on `stream`).  The paper has no counterpart: the predictor
 * picks the MTTKRP variant from tensor statistics.
 *   alto_nn_linear_forward : Y[n x dout] = act(X[n x din] W^T + b), W is
 *                            dout x din, act = ReLU when relu != 0.
 *   alto_nn_linear_backward: G = dY * act'(Y) (written to G, n x dout);
 *                            dW = G^T X, db = sum_rows G, dX = G W (dX may be
 *                            NULL).
 *   alto_nn_mse            : loss (device double) = sum(mask (P-T)^2) / norm,
 *                            dP = 2 mask (P-T) / norm; mask may be NULL.
 *   alto_nn_adam           : one Adam step (bias-corrected, step >= 1).
 */
alto_status alto_nn_linear_forward(const float *X, const float *W,
                                   const float *b, float *Y, int n, int din,
                                   int dout, int relu, void *stream);
alto_status alto_nn_linear_backward(const float *X, const float *W,
                                    const float *Y, const float *dY, float *G,
                                    float *dX, float *dW, float *db, int n,
                                    int din, int dout, int relu, void *stream);
alto_status alto_nn_mse(const float *P, const float *T, const float *mask,
                        float *dP, int64_t count, double norm, double *loss,
                        void *stream);
alto_status alto_nn_adam(float *param, const float *grad, float *m, float *v,
                         int64_t count, float lr, float beta1, float beta2,
                         float eps, int step, void *stream);

/* alto_set_variant -- override the MTTKRP variant of one mode. */
alto_status alto_set_variant(alto_t t, int mode, int variant);

/* alto_get_key_bytes -- bytes of one stored key in the streamed MTTKRP
 * format: the index and its flag bits in the fewest 32-bit words (4, 8, 12 or
 * 16 bytes; Sec. 4.2.3 stores native multiples, 32- and 96-bit words are the
 * packed widths), or the full word that alto_options.key_bits forces.
 * alto_export always widens keys to key_words 64-bit words. */
alto_status alto_get_key_bytes(alto_t t, int *bytes);

/* alto_set_parts -- segment count used by mode `mode`'s ATOMIC and WARPAGG
 * MTTKRPs (alto_mttkrp and batches planned afterwards): the line is cut into
 * nparts equal-nnz segments, 8 consecutive segments per thread block
 * (Sec. 3.2; L is a free parameter of the method).  0 restores the tensor's
 * own L; values above nnz are clamped to nnz.  SMEM and TEMP always use the
 * tensor's L (they read its per-segment intervals).  Errors: ALTO_EINVAL for
 * a NULL handle, a bad mode or a negative count. */
alto_status alto_set_parts(alto_t t, int mode, int64_t nparts);

/* alto_resolve_variant -- the accumulation variant an alto_mttkrp call of
 * this mode, rank and factor dtype runs when it asks for `variant`
 * (ALTO_VAR_AUTO: the per-mode override, else the reuse rule of Sec. 3.3
 * adapted to the GPU: reuse M/I_n <= 4 -> ATOMIC, else WARPAGG; SMEM is
 * never chosen automatically).  Shapes without a specialised kernel report
 * ATOMIC (the generic kernel).  *out receives one of
 * ALTO_VAR_ATOMIC..ALTO_VAR_GENERIC.  Host-only.  Errors: ALTO_EINVAL for a
 * NULL handle or output, a bad mode, rank, dtype or variant. */
alto_status alto_resolve_variant(alto_t t, int mode, int rank, alto_dtype fdtype, int variant, int *out);

/* alto_check -- synchronise `stream` and report a recorded device error. */
alto_status alto_check(alto_t t, void *stream);

/*
 * alto_layout_for_dims -- the index layout of Sec. 3.1 for given mode
 * lengths, computed on the host (no GPU needed).  Any output may be NULL.
 *   bits_per_mode : N entries; masks : N x 2 words (lo, hi);
 *   key_words     : 1 or 2; total_bits : sum of bits_per_mode (Eq. 1).
 * Errors: ALTO_EINVAL (bad N or length), ALTO_EOVERFLOW (above 128 bits or
 * above a forced 64-bit key).
 */
alto_status alto_layout_for_dims(int nmodes, const uint64_t *dims,
                                 int key_bits, int *bits_per_mode,
                                 uint64_t *masks, int *key_words,
                                 int *total_bits);

/*
 * alto_decode_host -- de-linearization (EXTRACT of Alg. 1) on the host with
 * the same precomputed masks the kernels use.  keys: count x key_words
 * uint64 (lo word first; flag bits are ignored); idx: count x N uint32
 * output (row-major).  Host memory only.
 */
alto_status alto_decode_host(int nmodes, const uint64_t *dims, int key_bits,
                             int64_t count, const uint64_t *keys,
                             uint32_t *idx);

/*
 * alto_profile -- enable (1) or disable (0) CUDA-event timing of this
 * handle's MTTKRP launches (output zeroing, the kernel and, for the Temp
 * variant, the pull pass), recorded on the launching stream.  Adds two event
 * records per MTTKRP call; off by default.
 */
alto_status alto_profile(alto_t t, int enable);

/*
 * alto_profile_read -- synchronise the recorded events and return, per mode,
 * the summed milliseconds (ms[N]) and number of timed MTTKRP calls
 * (calls[N]) since the previous read; then reset.  Either output may be NULL.
 */
alto_status alto_profile_read(alto_t t, double *ms, int64_t *calls);

/* alto_launch_count -- number of kernels the library has launched in this
 * process so far (all handles); the kernels of an alto_batch_run graph count
 * at every run. */
alto_status alto_launch_count(uint64_t *count);

/*
 * alto_linearize_noalloc -- the linearization and ordering stages of
 * alto_create (bit-level encode, stable sort) written into caller buffers,
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as
 * services that reserve all device memory for their own pool up front and
 * embedders whose device allocator belongs to another runtime.
 *
 *   idx   : host array of N DEVICE pointers to nnz indices (idx_bytes 4 or 8).
 *   keys  : device, nnz x key_words uint64 (key_words from
 *           alto_layout_for_dims; lo word first), ALTO order, no helper flags.
 *   perm  : device, nnz uint32, input position of every nonzero in ALTO order.
 * The sort's scratch lives in one fixed device array of about 5.3 MB that
 * every GPU which loads libalto holds until the process exits; nnz above
 * ALTO_NOALLOC_MAX_NNZ is rejected with ALTO_EINVAL.  Every call looks up
 * that array's device address in the current context.  All calls
 * share the array: calls that overlap on the GPU (other streams, other host
 * threads on the same device) race and must be serialised by the caller.
 * The call reads its status word back and synchronises `stream` at its end;
 * it returns ALTO_ERANGE when an index is out of range.
 */
#define ALTO_NOALLOC_MAX_NNZ 262144
alto_status alto_linearize_noalloc(int nmodes, const uint64_t *dims,
                                   int64_t nnz, const void *const *idx,
                                   int idx_bytes, uint64_t *keys,
                                   uint32_t *perm, void *stream);

/*
 * alto_batch_create -- plan many MTTKRPs (all modes of many tensors, of
 * uneven order and size) as one CUDA graph.  Item i is the mode-modes[i]
 * MTTKRP of tensors[i] with factors[i] (host array of that tensor's N device
 * pointers), rank ranks[i], factor dtype fdtype (shared by all items) and
 * output outs[i] (as for alto_mttkrp), using variants[i] (alto_variant, 0 =
 * automatic; NULL = all automatic).  Items of one kernel shape (order, key
 * width, rank, variant) run in one persistent launch over a device work list
 * of their thread-block units; the launches sit on parallel branches of the
 * graph (the costliest group first) so later groups fill the SMs that
 * earlier ones release; items without a
 * specialised kernel run on their own; the device-memory Temp variant is
 * replaced by warp aggregation.
 * The graph captures the given pointers: later runs read the factors' and
 * write the outputs' current contents.  Capture happens on `stream` (on a
 * private stream when `stream` is the legacy default stream, which cannot
 * be captured); the plan owns its device buffers.
 */
alto_status alto_batch_create(alto_batch_t *out, int count,
                              const alto_t *tensors, const int *modes,
                              const void *const *const *factors,
                              const int *ranks, alto_dtype fdtype,
                              void *const *outs, const int *variants,
                              void *stream);

/* alto_batch_run -- launch the plan's graph on `stream` (asynchronous). */
alto_status alto_batch_run(alto_batch_t b, void *stream);

/* alto_batch_info -- items, persistent group launches, stand-alone items,
 * and kernel launches per alto_batch_run (any pointer may be NULL). */
alto_status alto_batch_info(alto_batch_t b, int *items, int *groups,
                            int *single, int *kernels);

/* alto_batch_destroy -- free the plan.  NULL is accepted. */
alto_status alto_batch_destroy(alto_batch_t b);

/* alto_destroy -- free everything the handle owns.  NULL is accepted. */
alto_status alto_destroy(alto_t t);

/* Message for the last failure on the calling thread ("" if none). */
const char *alto_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ALTO_H */
