// Host-side internals of libalto: the tensor handle, the index layout and
// the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace alto {

// Index layout of one tensor (Sec. 3.1).
struct Layout {
  int N = 0;
  uint64_t dims[kMaxModes] = {};
  int nbits[kMaxModes] = {};
  int B = 0;                       // total index bits (Eq. 1 with whole bits)
  int KW = 1;                      // 64-bit words per key during generation and in exports
  int CW = 2;                      // 32-bit words per stored (MTTKRP) key: 1..4
  int pos[kMaxModes][32] = {};     // key bit of bit l of mode n
  uint64_t mask[kMaxModes][2] = {};
  int flag_bit[kMaxModes] = {};    // -1: no helper flag for the mode
  int hot_bit[kMaxModes] = {};     // -1: no hot-row flag for the mode
};

// Workspace of the CP-ALS driver, allocated on first use.
struct CpalsWork {
  int R = 0;
  alto_dtype fdtype = ALTO_F32;
  void* mt = nullptr;        // MTTKRP output, max I_n x R (FP32 or FP64)
  void* atmp = nullptr;      // unnormalised solve result, same size
  double* gram = nullptr;    // N x R x R
  double* vinv64 = nullptr;  // R x R
  float* vinv32 = nullptr;   // R x R
  double* colstat = nullptr; // R
  double* scal = nullptr;    // [0] inner product <X, model>, [1..] spare
  double* fits = nullptr;    // device fit per iteration
  int fits_cap = 0;
};

// Device-memory Temp variant (Alg. 2 literally): every thread-block unit u
// accumulates into its own Temp_u of (hi_u - lo_u + 1) x R elements, then a
// pull pass sums, for every output row b, the Temp_u of all units whose
// interval contains b.
struct TempPlan {
  int R = 0;
  size_t osz = 0;
  size_t temp_elems = 0;
  void* temp = nullptr;          // all Temp_u back to back
  uint64_t* toff = nullptr;      // element offset of Temp_u
  uint32_t* ulo = nullptr;       // interval start of unit u
  uint64_t* row_ptr = nullptr;   // CSR over output rows: covering units
  uint32_t* row_units = nullptr;
  bool built = false;
  bool feasible = false;
};

// Cap on the device-memory Temp of one mode.
constexpr size_t kTempCapBytes = size_t(4) << 30;

}  // namespace alto

struct alto_tensor_s {
  alto::Layout lay;
  int64_t M = 0;
  int64_t L = 0;             // equal-nnz line segments
  alto_dtype vdtype = ALTO_F32;
  // allocator
  void* (*alloc_fn)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  // device format (owned)
  uint64_t* keys = nullptr;   // M x KW, ALTO order, flags in spare bits (generation; freed when packed)
  uint32_t* ckeys = nullptr;  // M x CW stored keys for MTTKRP (aliases keys when CW == 2 KW)
  uint32_t* perm = nullptr;   // M, input position of each nonzero
  void* vals = nullptr;       // M values in ALTO order
  uint32_t* ivl = nullptr;    // L x N x 2 closed intervals
  uint32_t* hot[alto::kMaxModes] = {};  // hot rows per mode, hottest first
  int hot_n[alto::kMaxModes] = {};
  double hot_share[alto::kMaxModes] = {};  // sampled nonzeros in the hot rows / all samples
  void* hot_rep = nullptr;              // MTTKRP hot-row replicas (lazy)
  size_t hot_rep_bytes = 0;
  int* status = nullptr;      // device status word
  // statistics
  uint64_t distinct[alto::kMaxModes] = {};
  uint64_t max_ivl[alto::kMaxModes] = {};
  double reuse[alto::kMaxModes] = {};
  int variant[alto::kMaxModes] = {};
  int64_t mode_parts[alto::kMaxModes] = {};  // per-mode segment count of ATOMIC / WARPAGG (0: L)
  int gram_engine = 0;  // ALTO_GRAM_*: Gram matrices of CP-ALS on tensor cores (BF16) or CUDA cores
  double normX2 = 0.0;
  // Thread-block units (8 consecutive segments): union of their intervals
  // per mode, kept on the host (unit_lo / unit_hi) and as sorted widths.
  std::vector<uint32_t> unit_lo[alto::kMaxModes];
  std::vector<uint32_t> unit_hi[alto::kMaxModes];
  std::vector<uint32_t> unit_width_sorted[alto::kMaxModes];
  // device-memory Temp variant, per mode (built on first use)
  alto::TempPlan tp[alto::kMaxModes];
  alto::CpalsWork cp;
  // MTTKRP event timing (alto_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_mode;  // mode of the i-th recorded (start, stop) pair
  size_t ev_used = 0;        // pairs recorded since the last read

  // fraction of units whose output-mode interval has at most `rows` rows
  double unit_fit_frac(int mode, uint64_t rows) const {
    const std::vector<uint32_t>& w = unit_width_sorted[mode];
    if (w.empty()) return 1.0;
    const size_t k = static_cast<size_t>(
        std::upper_bound(w.begin(), w.end(), rows > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(rows)) -
        w.begin());
    return static_cast<double>(k) / static_cast<double>(w.size());
  }
};

namespace alto {

// process-wide count of kernel launches issued by the library
void note_launch(int k = 1);
uint64_t launch_total();

// MTTKRP event timing: record the start / stop of one timed call
cudaError_t prof_begin(alto_tensor_s* t, int mode, cudaStream_t s);
cudaError_t prof_end(alto_tensor_s* t, cudaStream_t s);

// allocation through the handle's allocator
void* dev_alloc(alto_tensor_s* t, size_t bytes);
void dev_free(alto_tensor_s* t, void* p);

// error reporting (thread-local message)
alto_status fail(alto_status code, const char* fmt, ...);

// sort.cu
// Key bits per radix-sort pass, and the passes radix_sort_pairs makes over
// nbits key bits (at least one, so that the position array is always written;
// the result lands in the first buffer pair after an even number of passes).
constexpr int kSortDigitBits = 8;
constexpr int sort_passes_for(int nbits) { return nbits > 0 ? (nbits + kSortDigitBits - 1) / kSortDigitBits : 1; }
// 32-bit words of sort scratch (tile counts, offsets, scan partials) for M keys
constexpr int64_t sort_scratch_words_for(int64_t M) {
  return 2 * (((M + 4095) / 4096) * 256) + ((((M + 4095) / 4096) * 256 + 8191) / 8192) + 64;
}
int64_t sort_scratch_words(int64_t M);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part,
                               cudaStream_t s);
cudaError_t radix_sort_pairs(uint64_t** keys, uint64_t** keys_alt, uint32_t** perm,
                             uint32_t** perm_alt, int64_t M, int KW, int nbits, uint32_t* scratch,
                             cudaStream_t s);

// gram_tc.cu: G += U^T U for BF16 U on the tensor cores (R in {8, 16, 32, 64}),
// and the CP-ALS form that first normalises the solved FP32 rows into U
bool gram_tc_supported(int R);
cudaError_t launch_gram_bf16_tc(const __nv_bfloat16* U, int64_t I, int R, double* G, int* status,
                                cudaStream_t s);
cudaError_t launch_normalize_gram_bf16_tc(const float* A, int64_t I, int R, const double* colstat, int use_max,
                                          double* lambda, __nv_bfloat16* U, double* G, const float* Mt,
                                          double* ip, int* status, cudaStream_t s);

// cpals.cu: G = U^T U (R x R FP64) through the chosen engine; synchronous
alto_status gram_any(const void* U, int64_t I, int R, alto_dtype dtype, int engine, double* G, cudaStream_t s);

// layout.cu (host only)
alto_status make_layout(int N, const uint64_t* dims, int key_bits, Layout* out);
void make_decode(const Layout& lay, const int* slot_mode, DecodeParams* dp);
void host_decode(const Layout& lay, const uint64_t* key, uint32_t* idx);

// encode.cu
struct IdxPtrs {
  const void* p[kMaxModes];
};
cudaError_t launch_encode(const Layout& lay, const IdxPtrs& idx, int idx_bytes, int64_t M,
                          uint64_t* keys, int* status, cudaStream_t s);
cudaError_t launch_pack_keys(const uint64_t* keys, int KW, uint32_t* out, int CW, int64_t M, cudaStream_t s);
cudaError_t launch_permute(const void* src, void* dst, const uint32_t* perm, int64_t M,
                           int elem_bytes, cudaStream_t s);
cudaError_t launch_sumsq(const uint64_t* keys, int KW, const void* vals, alto_dtype vd, int64_t M,
                         double* out, cudaStream_t s);
// Hot rows: every kHotSample-th nonzero is counted per row during the
// segment statistics pass; the rows with the largest sampled counts (at most
// kHotCap per mode) become the mode's hot list.
constexpr int kUnitSegs = 8;  // line segments per MTTKRP thread-block unit
constexpr int kHotSample = 16;
constexpr int kHotCap = 1024;
cudaError_t launch_segment_stats(const Layout& lay, const uint64_t* keys, int64_t M, int64_t L,
                                 uint32_t* ivl, uint32_t* const* first, uint32_t* const* last,
                                 uint32_t* const* cnt, cudaStream_t s);
cudaError_t launch_hot_hist(const uint32_t* cnt, uint64_t n, unsigned long long* hist, cudaStream_t s);
cudaError_t launch_hot_collect(const uint32_t* cnt, uint64_t n, uint32_t thr, uint32_t cap, uint32_t* out,
                               uint32_t* out_n, cudaStream_t s);
cudaError_t launch_count_touched(const uint32_t* first, uint64_t n, unsigned long long* out,
                                 cudaStream_t s);
cudaError_t launch_max_interval(const uint32_t* ivl, int64_t L, int N, unsigned long long* out,
                                cudaStream_t s);
cudaError_t launch_set_flags(const Layout& lay, uint64_t* keys, int64_t M,
                             uint32_t* const* first, uint32_t* const* last,
                             uint32_t* const* hotmap, cudaStream_t s);
cudaError_t launch_hot_map(const uint32_t* rows, int n, uint32_t* map, cudaStream_t s);

// mttkrp.cu
struct MttkrpLaunch;
alto_status run_mttkrp(alto_tensor_s* t, int mode, const void* const* factors, int R,
                       alto_dtype fdtype, void* out, int variant, cudaStream_t s);

// mttkrp_temp.cu
cudaError_t launch_temp_variant(alto_tensor_s* t, const MttkrpLaunch& l, alto_dtype fdtype,
                                size_t osz, cudaStream_t s);
alto_status build_temp_plan(alto_tensor_s* t, int mode, int R, size_t osz, cudaStream_t s);
void free_temp_plan(alto_tensor_s* t, int mode);

// cpals.cu
alto_status run_cpals(alto_tensor_s* t, int R, int iters, void* const* factors, alto_dtype fdtype,
                      double* lambda, double* fit, cudaStream_t s);

}  // namespace alto
