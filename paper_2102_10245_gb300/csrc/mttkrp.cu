// Host side of alto_mttkrp: argument checks, slot order, variant choice and
// dispatch to the per-dtype kernel instantiations.
#include <algorithm>

#include "mttkrp_kernels.cuh"

namespace alto {

namespace {

constexpr size_t kSmemTempBytes = 96 * 1024;  // shared Temp budget per block


int device_sms() {
  static int cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = s > 0 ? s : 1;
  }
  return cached[dev];
}

int smem_rows_for(const alto_tensor_s* t, int mode, int R, size_t osz) {
  size_t rows = kSmemTempBytes / (static_cast<size_t>(R) * osz);
  if (rows > t->lay.dims[mode]) rows = static_cast<size_t>(t->lay.dims[mode]);
  return static_cast<int>(rows);
}

}  // namespace

cudaError_t mttkrp_launch(alto_tensor_s* t, int mode, const void* const* factors, int R,
                          alto_dtype fdtype, void* out, int variant, size_t osz, cudaStream_t s);

// The Sec. 3.3 rule adapted to the GPU: fiber reuse M / I_n above 4 means
// buffered accumulation, realised as warp-level run aggregation in registers
// with replicated hot rows; reuse of at most 4 means direct atomics.  The
// shared-memory Temp (SMEM) is left to explicit choice: shared-memory FP32
// atomics are emulated on this GPU, and SMEM measured slower than WARPAGG
// even where the unit intervals fit (2.4x on a 100-row mode).
int auto_variant(const alto_tensor_s* t, int mode, int R, size_t osz) {
  (void)R;
  (void)osz;
  return t->reuse[mode] <= 4.0 ? ALTO_VAR_ATOMIC : ALTO_VAR_WARPAGG;
}

alto_status check_mttkrp_args(const alto_tensor_s* t, int mode, const void* const* factors, int R,
                              alto_dtype fdtype, const void* out, int variant) {
  const Layout& lay = t->lay;
  const int N = lay.N;
  if (mode < 0 || mode >= N) return fail(ALTO_EINVAL, "mode %d outside [0, %d)", mode, N);
  if (R < 1) return fail(ALTO_EINVAL, "rank %d < 1", R);
  if (out == nullptr || factors == nullptr) return fail(ALTO_EINVAL, "null factors or output");
  for (int m = 0; m < N; ++m)
    if (m != mode && factors[m] == nullptr) return fail(ALTO_EINVAL, "factor %d is null", m);
  if (fdtype == ALTO_F64) {
    if (t->vdtype != ALTO_F64) return fail(ALTO_EINVAL, "FP64 factors need FP64 values");
  } else if (fdtype == ALTO_F32 || fdtype == ALTO_BF16) {
    if (t->vdtype != ALTO_F32 && t->vdtype != ALTO_BF16)
      return fail(ALTO_EINVAL, "FP32/BF16 factors need FP32 or BF16 values");
  } else {
    return fail(ALTO_EINVAL, "bad factor dtype %d", static_cast<int>(fdtype));
  }
  if (variant < ALTO_VAR_AUTO || variant > ALTO_VAR_GENERIC) return fail(ALTO_EINVAL, "bad variant %d", variant);
  return ALTO_OK;
}

// The variant an MTTKRP call runs: the call's, else the tensor's per-mode
// override, else the automatic rule.
int resolve_variant(const alto_tensor_s* t, int mode, int R, size_t osz, int variant) {
  int v = variant != ALTO_VAR_AUTO ? variant : t->variant[mode];
  if (v == ALTO_VAR_AUTO) v = auto_variant(t, mode, R, osz);
  return v;
}

// Segment count of an MTTKRP: the per-mode override for the ATOMIC and
// WARPAGG policies (they use the segments only to cut the line into
// thread-block units), else the tensor's L (SMEM and TEMP read the segments'
// intervals).  At most M, at least 1.
int64_t mttkrp_parts(const alto_tensor_s* t, int mode, int variant) {
  const int64_t p = t->mode_parts[mode];
  if (p <= 0 || !(variant == ALTO_VAR_ATOMIC || variant == ALTO_VAR_WARPAGG)) return t->L;
  return p < t->M ? p : (t->M > 0 ? t->M : 1);
}

// Arguments common to every variant.
void fill_launch(const alto_tensor_s* t, int mode, const void* const* factors, int R, void* out,
                 MttkrpLaunch* l) {
  const Layout& lay = t->lay;
  const int N = lay.N;
  int slot_mode[kMaxModes];
  int k = 0;
  for (int m = 0; m < N; ++m)
    if (m != mode) slot_mode[k++] = m;
  slot_mode[k] = mode;
  make_decode(lay, slot_mode, &l->args.dp);
  l->args.keys = t->ckeys;
  l->args.vals = t->vals;
  l->args.vbf16 = t->vdtype == ALTO_BF16 ? 1 : 0;
  l->args.M = t->M;
  l->args.L = t->L;
  for (int sl = 0; sl < N; ++sl) l->args.f[sl] = factors[slot_mode[sl]];
  l->args.out = out;
  l->args.R = R;
  l->args.out_mode = mode;
  l->args.ivl = t->ivl;
  l->N = N;
  l->W32 = lay.CW;
  l->sms = device_sms();
}

size_t smem_temp_bytes(const alto_tensor_s* t, int mode, int R, size_t osz, int* rows_out) {
  const int rows = smem_rows_for(t, mode, R, osz);
  *rows_out = rows;
  return static_cast<size_t>(rows) * R * osz + static_cast<size_t>((rows + 31) / 32) * 4;
}

alto_status run_mttkrp(alto_tensor_s* t, int mode, const void* const* factors, int R,
                       alto_dtype fdtype, void* out, int variant, cudaStream_t s) {
  alto_status st = check_mttkrp_args(t, mode, factors, R, fdtype, out, variant);
  if (st != ALTO_OK) return st;
  const size_t osz = fdtype == ALTO_F64 ? 8 : 4;
  cudaError_t e = prof_begin(t, mode, s);
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "profiling event: %s", cudaGetErrorString(e));
  e = mttkrp_launch(t, mode, factors, R, fdtype, out, variant, osz, s);
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "MTTKRP launch: %s", cudaGetErrorString(e));
  e = prof_end(t, s);
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "profiling event: %s", cudaGetErrorString(e));
  return ALTO_OK;
}

cudaError_t mttkrp_launch(alto_tensor_s* t, int mode, const void* const* factors, int R,
                          alto_dtype fdtype, void* out, int variant, size_t osz, cudaStream_t s) {
  const Layout& lay = t->lay;
  const int N = lay.N;
  cudaError_t e = cudaMemsetAsync(out, 0, static_cast<size_t>(lay.dims[mode]) * R * osz, s);
  if (e != cudaSuccess) return e;
  if (t->M == 0) return cudaSuccess;

  int v = resolve_variant(t, mode, R, osz, variant);
  MttkrpLaunch l{};
  fill_launch(t, mode, factors, R, out, &l);
  if (v == ALTO_VAR_TEMP) return launch_temp_variant(t, l, fdtype, osz, s);
  if (v == ALTO_VAR_GENERIC) {  // the rank- and order-generic kernel on request
    l.variant = v;
    l.generic = true;
    return mttkrp_dispatch(l, fdtype, s);
  }
  if (!mttkrp_specialised(N, R)) v = ALTO_VAR_ATOMIC;  // the generic kernel
  l.variant = v;
  l.args.L = mttkrp_parts(t, mode, v);
  const size_t fsz = fdtype == ALTO_F64 ? 8 : (fdtype == ALTO_F32 ? 4 : 2);
  l.fused = (v == ALTO_VAR_ATOMIC || v == ALTO_VAR_WARPAGG) && mttkrp_specialised(N, R) &&
            fused_ok(N, R, fsz, l.args.f, out, osz, lay.dims[mode]);
  int H = 0;
  if (v == ALTO_VAR_WARPAGG && lay.dims[mode] <= (1ull << 31) && mttkrp_specialised(N, R)) {
    H = t->hot_n[mode];
    if (H > 0) {
      // replicas of the hot rows: kHotReplicas x kHotCap x R, kept in the handle
      const size_t need = static_cast<size_t>(kHotReplicas) * kHotCap * R * osz;
      if (t->hot_rep_bytes < need) {
        dev_free(t, t->hot_rep);
        t->hot_rep = dev_alloc(t, need);
        t->hot_rep_bytes = t->hot_rep ? need : 0;
        if (t->hot_rep == nullptr) return cudaErrorMemoryAllocation;
      }
      e = cudaMemsetAsync(t->hot_rep, 0, static_cast<size_t>(kHotReplicas) * H * R * osz, s);
      if (e != cudaSuccess) return e;
      int bits = 1;
      while ((1 << bits) < 2 * H) ++bits;
      l.args.hot = t->hot[mode];
      l.args.hot_n = H;
      l.args.hot_bits = bits;
      l.args.hot_key_bit = lay.hot_bit[mode];
      l.args.hot_rep = t->hot_rep;
      l.smem_dyn = static_cast<size_t>(2) * (1u << bits) * sizeof(uint32_t);
    }
  }
  if (v == ALTO_VAR_SMEM) {
    int rows = 0;
    l.smem_dyn = smem_temp_bytes(t, mode, R, osz, &rows);
    l.args.smem_rows = rows;
  }
  e = mttkrp_dispatch(l, fdtype, s);
  if (e != cudaSuccess || H == 0) return e;
  const int total = H * R;
  const unsigned g = static_cast<unsigned>((total + 255) / 256);
  if (osz == 8)
    hot_reduce_kernel<double><<<g, 256, 0, s>>>(static_cast<const double*>(t->hot_rep), t->hot[mode], H, R,
                                                kHotReplicas, static_cast<double*>(out));
  else
    hot_reduce_kernel<float><<<g, 256, 0, s>>>(static_cast<const float*>(t->hot_rep), t->hot[mode], H, R,
                                               kHotReplicas, static_cast<float*>(out));
  note_launch();
  return cudaGetLastError();
}

}  // namespace alto

using namespace alto;

extern "C" alto_status alto_resolve_variant(alto_t t, int mode, int rank, alto_dtype fdtype, int variant,
                                            int* out) {
  if (t == nullptr || out == nullptr) return fail(ALTO_EINVAL, "null argument");
  if (mode < 0 || mode >= t->lay.N) return fail(ALTO_EINVAL, "mode %d outside [0, %d)", mode, t->lay.N);
  if (rank < 1) return fail(ALTO_EINVAL, "rank %d < 1", rank);
  if (variant < ALTO_VAR_AUTO || variant > ALTO_VAR_GENERIC) return fail(ALTO_EINVAL, "bad variant %d", variant);
  if (fdtype != ALTO_F64 && fdtype != ALTO_F32 && fdtype != ALTO_BF16)
    return fail(ALTO_EINVAL, "bad factor dtype %d", static_cast<int>(fdtype));
  const size_t osz = fdtype == ALTO_F64 ? 8 : 4;
  int v = resolve_variant(t, mode, rank, osz, variant);
  if (v != ALTO_VAR_TEMP && v != ALTO_VAR_GENERIC && !mttkrp_specialised(t->lay.N, rank)) v = ALTO_VAR_ATOMIC;
  *out = v;
  return ALTO_OK;
}
