// MTTKRP over the ALTO format (Sec. 2.2, Alg. 1-2), GPU kernel family.
//
// Work split.  The ordered nonzeros are cut into L equal-nnz line segments
// (Sec. 3.2); a thread block takes a unit of 8 consecutive segments, and its
// 8 warps walk the unit in interleaved chunks of 32 nonzeros (warp w takes
// chunks w, w+8, ...), so the rows a block touches at any moment come from a
// short stretch of the line and stay in L1 / L2.  Per chunk:
//   1. each lane de-linearizes one nonzero (bit-level compress per 32-bit key
//      word, EXTRACT of Alg. 2); the next chunk's key and value are already
//      being fetched;
//   2. the decoded tuple (N indices + value) is staged in shared memory;
//   3. groups of LPN lanes own one staged nonzero at a time, each lane CPL
//      columns in VEC-element pieces; the gathers of the next position are
//      issued before the current position's arithmetic (Hadamard product of
//      the N-1 input rows, scaled by the value, packed FP32x2 math).
//
// Output accumulation policies (Alg. 2 and the Sec. 3.3 rule):
//   ATOMIC  every nonzero adds its row into the output with vector atomics
//           (the ATOMIC branch of Alg. 2);
//   WARPAGG the chunk is reordered by output row inside the warp (match on
//           the row, prefix over the matched sets) so equal rows are
//           consecutive; a group sums a run in registers and adds it with one
//           vector atomic.  Rows of the mode's hot list (the rows with the
//           most nonzeros; their elements carry a hot flag in a spare key
//           bit) are found in a shared-memory hash table while staging and
//           added into one of kHotReplicas copies of the hot rows (chosen by
//           block), which a small pass sums into the output afterwards: heavy
//           rows no longer serialise on one L2 slice;
//   SMEM    the unit's Temp lives in shared memory over the union of its
//           segments' output-mode intervals (Temp_l of Alg. 2), filled with
//           shared-memory atomics and flushed once per touched row; a unit
//           whose interval does not fit falls back to WARPAGG;
//   TEMP    as WARPAGG but into the unit's own Temp_u in device memory; a pull
//           pass (mttkrp_temp.cu) then reduces the Temps into the output.
// All policies compute the same sums; only the rounding order differs.
#pragma once

#include <type_traits>

#include "internal.h"

namespace alto {

enum Policy { kAtomic = ALTO_VAR_ATOMIC, kWarpAgg = ALTO_VAR_WARPAGG, kSmem = ALTO_VAR_SMEM, kTemp = ALTO_VAR_TEMP };

// ---------------------------------------------------------------------------
// factor element traits: loads of VEC elements per lane, accumulation type
// AT; gathered rows are held as RT words of PACK elements each (BF16 rows
// stay packed in registers and are widened where they are used).  BF16 rows
// are loaded 8 bytes per lane: with 16-byte loads a warp instruction touched
// twice as many rows and the kernel ran 1.6x slower on GB300.
template <typename FT>
struct FTraits;
template <>
struct FTraits<float> {
  static constexpr int VEC = 4;
  static constexpr int PACK = 1;
  using AT = float;
  using VT = float;
  using RT = float;
};
template <>
struct FTraits<double> {
  static constexpr int VEC = 2;
  static constexpr int PACK = 1;
  using AT = double;
  using VT = double;
  using RT = double;
};
template <>
struct FTraits<__nv_bfloat16> {
  static constexpr int VEC = 4;
  static constexpr int PACK = 2;
  using AT = float;
  using VT = float;
  using RT = uint32_t;
};

// Column layout of one nonzero's row across its lane group: lane c of the
// group owns the VEC-element pieces at columns c*VEC + q*STRIDE, q < PAIRS.
// One piece per lane up to 32 lanes keeps every warp-wide access at one L1
// wavefront per row (the SM's L1 / shared path moves about 128 bytes per
// clock, which bounds the gathers).
template <int R, typename FT>
struct Cols {
  static constexpr int VEC = FTraits<FT>::VEC;
  static constexpr int PAIRS = (R / VEC > 32) ? R / VEC / 32 : 1;
  static constexpr int LPN = R / (VEC * PAIRS);  // lanes per nonzero
  static constexpr int STRIDE = R / PAIRS;
  static constexpr int CPL = VEC * PAIRS;        // columns per lane
  static_assert(LPN >= 1 && LPN <= 32 && 32 % LPN == 0, "rank / vector width");
};

template <typename FT>
__device__ __forceinline__ void load_vec(const FT* p, typename FTraits<FT>::RT* v);

template <>
__device__ __forceinline__ void load_vec<float>(const float* p, float* v) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}

template <>
__device__ __forceinline__ void load_vec<double>(const double* p, double* v) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = a.x;
  v[1] = a.y;
}

template <>
__device__ __forceinline__ void load_vec<__nv_bfloat16>(const __nv_bfloat16* p, uint32_t* v) {
  const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
  v[0] = a.x;
  v[1] = a.y;
}

// two BF16 values packed in a word (element 0 in the low half) as FP32: a
// BF16 value is the upper 16 bits of the FP32 value with the same bits
__device__ __forceinline__ float2 widen_bf16x2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// elementwise helpers, packed FP32x2 where the accumulation type is float
template <int K>
__device__ __forceinline__ void scale_into(float* t, float v, const float* a) {
  const float2 v2 = make_float2(v, v);
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    const float2 r = __fmul2_rn(v2, make_float2(a[e], a[e + 1]));
    t[e] = r.x;
    t[e + 1] = r.y;
  }
}
template <int K>
__device__ __forceinline__ void scale_into(float* t, float v, const uint32_t* a) {
  const float2 v2 = make_float2(v, v);
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    const float2 r = __fmul2_rn(v2, widen_bf16x2(a[e / 2]));
    t[e] = r.x;
    t[e + 1] = r.y;
  }
}
template <int K>
__device__ __forceinline__ void mul_into(float* t, const uint32_t* a) {
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    const float2 r = __fmul2_rn(make_float2(t[e], t[e + 1]), widen_bf16x2(a[e / 2]));
    t[e] = r.x;
    t[e + 1] = r.y;
  }
}
template <int K>
__device__ __forceinline__ void fma_into(float* acc, const float* t, const uint32_t* a) {
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    const float2 r = __ffma2_rn(make_float2(t[e], t[e + 1]), widen_bf16x2(a[e / 2]), make_float2(acc[e], acc[e + 1]));
    acc[e] = r.x;
    acc[e + 1] = r.y;
  }
}
template <int K>
__device__ __forceinline__ void scale_into(double* t, double v, const double* a) {
#pragma unroll
  for (int e = 0; e < K; ++e) t[e] = v * a[e];
}
template <int K>
__device__ __forceinline__ void mul_into(float* t, const float* a) {
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    const float2 r = __fmul2_rn(make_float2(t[e], t[e + 1]), make_float2(a[e], a[e + 1]));
    t[e] = r.x;
    t[e + 1] = r.y;
  }
}
template <int K>
__device__ __forceinline__ void mul_into(double* t, const double* a) {
#pragma unroll
  for (int e = 0; e < K; ++e) t[e] *= a[e];
}
template <int K>
__device__ __forceinline__ void fma_into(float* acc, const float* t, const float* a) {
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    const float2 r =
        __ffma2_rn(make_float2(t[e], t[e + 1]), make_float2(a[e], a[e + 1]), make_float2(acc[e], acc[e + 1]));
    acc[e] = r.x;
    acc[e + 1] = r.y;
  }
}
template <int K>
__device__ __forceinline__ void fma_into(double* acc, const double* t, const double* a) {
#pragma unroll
  for (int e = 0; e < K; ++e) acc[e] = fma(t[e], a[e], acc[e]);
}

// VEC accumulators into global memory with vector atomics
template <int VEC>
__device__ __forceinline__ void red_vec(float* out, const float* v) {
  static_assert(VEC % 4 == 0, "FP32 accumulators flush in fours");
#pragma unroll
  for (int j = 0; j < VEC; j += 4) red_add_v4(out + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
}
template <int VEC>
__device__ __forceinline__ void red_vec(double* out, const double* v) {
#pragma unroll
  for (int j = 0; j < VEC; ++j) red_add_f64(out + j, v[j]);
}

struct MttkrpArgs {
  const uint32_t* keys;      // stored keys, W32 words each
  const void* vals;          // FP64 when the factors are FP64, else FP32 or BF16 (vbf16)
  int64_t M;
  int64_t L;                 // line segments
  const void* f[kMaxModes];  // factor of each decode slot; slot N-1 is the output mode
  void* out;
  int R;
  int out_mode;              // mode of the output (column of the interval table)
  const uint32_t* ivl;       // L x N x 2 segment intervals
  int smem_rows;             // SMEM: rows of the shared Temp
  void* temp;                // TEMP: all Temp_u back to back
  const uint64_t* toff;      // TEMP: element offset of Temp_u
  const uint32_t* ulo;       // TEMP: interval start of unit u
  const uint32_t* hot;       // WARPAGG: hot rows of the output mode
  int hot_n;                 // WARPAGG: hot rows in the table (0: none)
  int hot_bits;              // WARPAGG: log2 of the hash table size
  int hot_key_bit;           // WARPAGG: key bit flagging hot output rows, or -1
  void* hot_rep;             // WARPAGG: kHotReplicas x hot_n x R accumulators
  int vbf16;                 // values stored as BF16 (FP32 / BF16 factors only)
  DecodeParams dp;
};

constexpr uint32_t kHotEmpty = 0xffffffffu;
constexpr int kHotReplicas = 32;  // copies of the hot rows (block b adds into copy b % 32)

__device__ __forceinline__ uint32_t hot_hash(uint32_t row, int bits) {
  return (row * 0x9E3779B1u) >> (32 - bits);
}

// slot of `row` in the block's hot table, or -1
__device__ __forceinline__ int hot_lookup(const uint32_t* keys, const uint32_t* idx, uint32_t row, int bits) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t h = hot_hash(row, bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {  // at most half full: an empty slot ends it early
    const uint32_t k = keys[h];
    if (k == row) return static_cast<int>(idx[h]);
    if (k == kHotEmpty) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
// Positions whose factor-row gathers are in flight ahead of the sum.  Depths 2
// and 3 (with the register budget they need) measured no faster on GB300:
// the L1 data path, not the latency of single gathers, bounds the kernel.
constexpr int kGatherDepth = 1;
static_assert(sizeof(MttkrpArgs) % 4 == 0, "MttkrpArgs is copied as 32-bit words");

// Value x of the tensor as the accumulation's value type: FP64 values for
// FP64 factors; FP32 or BF16 values (widened exactly) otherwise.  Streamed
// once, so loaded with the evict-first hint.  Both 32-bit forms take one
// 4-byte load and no branch: FP32 reads word x; BF16 reads word x/2, whose
// low half holds the even element and high half the odd one.  The load and
// the widening are separate steps: a pipeline that prefetches the next
// chunk's values keeps the raw word and widens it when the chunk is used, so
// the load's latency stays hidden (widening right after the load made every
// prefetch wait for its data: 4.08 against 3.42 ms per mode).  The value
// buffer is padded past M, so the word of the last odd-count BF16 element is
// in bounds.
template <typename VT>
struct VRaw {
  using T = uint32_t;
};
template <>
struct VRaw<double> {
  using T = double;
};

template <typename VT>
__device__ __forceinline__ typename VRaw<VT>::T load_value_raw(const MttkrpArgs& a, int64_t x) {
  if constexpr (std::is_same_v<VT, double>) {
    return __ldcs(static_cast<const double*>(a.vals) + x);
  } else {
    return __ldcs(static_cast<const unsigned int*>(a.vals) + (x >> a.vbf16));
  }
}

template <typename VT>
__device__ __forceinline__ VT value_of(const MttkrpArgs& a, typename VRaw<VT>::T w, int64_t x) {
  if constexpr (std::is_same_v<VT, double>) {
    return w;
  } else {
    const uint32_t h = static_cast<uint32_t>(a.vbf16);  // 0 or 1
    const uint32_t odd = static_cast<uint32_t>(x) & h;
    const uint32_t lsh = (h & ~odd) << 4;      // 16 for an even BF16 element
    const uint32_t keep = ~(odd * 0xffffu);    // 0xffff0000 for an odd one
    return __uint_as_float((w << lsh) & keep);
  }
}

template <typename VT>
__device__ __forceinline__ VT load_value(const MttkrpArgs& a, int64_t x) {
  return value_of<VT>(a, load_value_raw<VT>(a, x), x);
}

// staged tuple: N indices and the value, padded to 16-byte words
template <int N, typename VT>
struct Stage {
  static constexpr int WORDS_RAW = N + static_cast<int>(sizeof(VT) / 4);
  static constexpr int W4 = (WORDS_RAW + 3) / 4;  // uint4 per entry
};

template <int N, typename VT>
__device__ __forceinline__ void stage_store(uint4* slot, const uint32_t* id, VT v) {
  uint32_t w[Stage<N, VT>::W4 * 4];
#pragma unroll
  for (int s = 0; s < N; ++s) w[s] = id[s];
  memcpy(&w[N], &v, sizeof(VT));
#pragma unroll
  for (int s = N + static_cast<int>(sizeof(VT) / 4); s < Stage<N, VT>::W4 * 4; ++s) w[s] = 0;
#pragma unroll
  for (int q = 0; q < Stage<N, VT>::W4; ++q) slot[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

template <int N, typename VT>
struct Pos {
  uint32_t id[N];
  VT v;
};

template <int N, typename VT>
__device__ __forceinline__ Pos<N, VT> stage_load(const uint4* slot) {
  uint32_t w[Stage<N, VT>::W4 * 4];
#pragma unroll
  for (int q = 0; q < Stage<N, VT>::W4; ++q) {
    const uint4 x = slot[q];
    w[4 * q] = x.x;
    w[4 * q + 1] = x.y;
    w[4 * q + 2] = x.z;
    w[4 * q + 3] = x.w;
  }
  Pos<N, VT> p;
#pragma unroll
  for (int s = 0; s < N; ++s) p.id[s] = w[s];
  memcpy(&p.v, &w[N], sizeof(VT));
  return p;
}

// gathered input rows of one position: (N-1) x CPL values in RT words
template <int N, int R, typename FT>
struct Rows {
  typename FTraits<FT>::RT u[N > 1 ? N - 1 : 1][Cols<R, FT>::CPL / FTraits<FT>::PACK];
};

template <int N, int R, typename FT, typename VT>
__device__ __forceinline__ void gather(const MttkrpArgs& a, const Pos<N, VT>& p, int c, Rows<N, R, FT>& r) {
  using C = Cols<R, FT>;
#pragma unroll
  for (int s = 0; s < N - 1; ++s) {
    const FT* row = static_cast<const FT*>(a.f[s]) + static_cast<size_t>(p.id[s]) * R + c * C::VEC;
#pragma unroll
    for (int q = 0; q < C::PAIRS; ++q) load_vec<FT>(row + q * C::STRIDE, &r.u[s][q * C::VEC / FTraits<FT>::PACK]);
  }
}

// Exact FP32 products of two packed BF16 pairs (an 8-bit by 8-bit significand
// product fits FP32's 24 bits), by the mixed-precision FMA with a zero addend.
__device__ __forceinline__ float2 bf16x2_mul_exact(uint32_t a, uint32_t b) {
  float lo, hi;
  asm("{\n\t.reg .b16 al, ah, bl, bh;\n\t"
      "mov.b32 {al, ah}, %2;\n\t"
      "mov.b32 {bl, bh}, %3;\n\t"
      "fma.rn.f32.bf16 %0, al, bl, 0f00000000;\n\t"
      "fma.rn.f32.bf16 %1, ah, bh, 0f00000000;\n\t}"
      : "=f"(lo), "=f"(hi)
      : "r"(a), "r"(b));
  return make_float2(lo, hi);
}

// BF16 rows: the first two rows' product is formed exactly from the packed
// words, the other rows are widened and multiplied in FP32, and the value
// scales last: pr = u_0 * u_1 * ... * u_{N-2} (FP32), so that
// t = v * pr and acc += v * pr are single packed FP32 operations.
template <int N, int R>
__device__ __forceinline__ void bf16_row_product(const Rows<N, R, __nv_bfloat16>& r, float* pr) {
  constexpr int K = Cols<R, __nv_bfloat16>::CPL;
#pragma unroll
  for (int e = 0; e < K; e += 2) {
    float2 x = bf16x2_mul_exact(r.u[0][e / 2], r.u[1][e / 2]);
#pragma unroll
    for (int s = 2; s < N - 1; ++s) x = __fmul2_rn(x, widen_bf16x2(r.u[s][e / 2]));
    pr[e] = x.x;
    pr[e + 1] = x.y;
  }
}

// t = v * prod_s u_s
template <int N, int R, typename FT, typename VT>
__device__ __forceinline__ void product(const Pos<N, VT>& p, const Rows<N, R, FT>& r,
                                        typename FTraits<FT>::AT* t) {
  using AT = typename FTraits<FT>::AT;
  constexpr int K = Cols<R, FT>::CPL;
  if constexpr (std::is_same_v<FT, __nv_bfloat16> && N >= 3) {
    bf16_row_product<N, R>(r, t);
    const float2 v2 = make_float2(static_cast<float>(p.v), static_cast<float>(p.v));
#pragma unroll
    for (int e = 0; e < K; e += 2) {
      const float2 x = __fmul2_rn(v2, make_float2(t[e], t[e + 1]));
      t[e] = x.x;
      t[e + 1] = x.y;
    }
  } else if constexpr (N == 1) {
#pragma unroll
    for (int e = 0; e < K; ++e) t[e] = static_cast<AT>(p.v);
  } else {
    scale_into<K>(t, static_cast<AT>(p.v), r.u[0]);
#pragma unroll
    for (int s = 1; s < N - 1; ++s) mul_into<K>(t, r.u[s]);
  }
}

// acc += v * prod_s u_s
template <int N, int R, typename FT, typename VT>
__device__ __forceinline__ void accumulate(const Pos<N, VT>& p, const Rows<N, R, FT>& r,
                                           typename FTraits<FT>::AT* acc) {
  using AT = typename FTraits<FT>::AT;
  constexpr int K = Cols<R, FT>::CPL;
  AT t[K];
  if constexpr (std::is_same_v<FT, __nv_bfloat16> && N >= 3) {
    bf16_row_product<N, R>(r, t);
    const float2 v2 = make_float2(static_cast<float>(p.v), static_cast<float>(p.v));
#pragma unroll
    for (int e = 0; e < K; e += 2) {
      const float2 x = __ffma2_rn(v2, make_float2(t[e], t[e + 1]), make_float2(acc[e], acc[e + 1]));
      acc[e] = x.x;
      acc[e + 1] = x.y;
    }
  } else if constexpr (N <= 2) {
    product<N, R, FT>(p, r, t);
#pragma unroll
    for (int e = 0; e < K; ++e) acc[e] += t[e];
  } else {
    scale_into<K>(t, static_cast<AT>(p.v), r.u[0]);
#pragma unroll
    for (int s = 1; s < N - 2; ++s) mul_into<K>(t, r.u[s]);
    fma_into<K>(acc, t, r.u[N - 2]);
  }
}

// flush a lane's CPL accumulators of one row into a dense row-major
// destination (output or Temp) with vector atomics
template <int R, typename FT>
__device__ __forceinline__ void flush_global(typename FTraits<FT>::AT* rowp, int c,
                                             const typename FTraits<FT>::AT* acc) {
  using C = Cols<R, FT>;
#pragma unroll
  for (int q = 0; q < C::PAIRS; ++q) red_vec<C::VEC>(rowp + c * C::VEC + q * C::STRIDE, acc + q * C::VEC);
}

template <int R, typename FT>
__device__ __forceinline__ void flush_shared(typename FTraits<FT>::AT* rowp, int c,
                                             const typename FTraits<FT>::AT* acc) {
  using C = Cols<R, FT>;
#pragma unroll
  for (int q = 0; q < C::PAIRS; ++q)
#pragma unroll
    for (int e = 0; e < C::VEC; ++e) atomicAdd(rowp + c * C::VEC + q * C::STRIDE + e, acc[q * C::VEC + e]);
}

// ---------------------------------------------------------------------------
// Per-block state of one MTTKRP (hot-row table, replica).
template <typename AT>
struct BlockState {
  int H;
  AT* hdata;
  uint32_t* hkeys;
  uint32_t* hidx;
};

// Build the block's hot-row hash table in shared memory (WARPAGG).
template <typename AT, int R>
__device__ __forceinline__ BlockState<AT> hot_table(const MttkrpArgs& a, unsigned char* dyn, int replica) {
  BlockState<AT> st{0, nullptr, nullptr, nullptr};
  st.H = a.hot_n;
  if (st.H > 0) {
    const int TS = 1 << a.hot_bits;
    st.hdata = static_cast<AT*>(a.hot_rep) + static_cast<size_t>(replica) * st.H * R;
    st.hkeys = reinterpret_cast<uint32_t*>(dyn);
    st.hidx = st.hkeys + TS;
    for (int i = threadIdx.x; i < TS; i += kThreads) st.hkeys[i] = kHotEmpty;
    __syncthreads();
    const uint32_t mask = static_cast<uint32_t>(TS - 1);
    for (int i = threadIdx.x; i < st.H; i += kThreads) {
      const uint32_t row = a.hot[i];
      uint32_t h = hot_hash(row, a.hot_bits);
      for (int probe = 0; probe < TS; ++probe) {
        if (atomicCAS(st.hkeys + h, kHotEmpty, row) == kHotEmpty) {
          st.hidx[h] = static_cast<uint32_t>(i);
          break;
        }
        h = (h + 1) & mask;
      }
    }
  }
  __syncthreads();
  return st;
}

// One thread-block unit (8 consecutive segments) of one MTTKRP.  All threads
// of the block call it together.
template <int N, int W32, int R, typename FT, int POL>
__device__ __forceinline__ void process_unit(const MttkrpArgs& a, int64_t u,
                                             const BlockState<typename FTraits<FT>::AT>& st,
                                             uint4 (*s_stage)[32][Stage<N, typename FTraits<FT>::VT>::W4],
                                             uint32_t* s_lorows, unsigned char* dyn) {
  using AT = typename FTraits<FT>::AT;
  using VT = typename FTraits<FT>::VT;
  using C = Cols<R, FT>;
  constexpr int LPN = C::LPN;
  constexpr int PER = LPN;             // staged positions per group (32 / groups)
  constexpr int K = C::CPL;
  constexpr bool AGG = POL != kAtomic;  // reorder by output row before the gathers
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / LPN, c = lane % LPN;
  const uint32_t lt = lanemask_lt();
  AT* out = static_cast<AT*>(a.out);
  const int H = st.H;

  const int64_t useg1 = (u + 1) * kUnitSegs < a.L ? (u + 1) * kUnitSegs : a.L;
  const int64_t ub = seg_begin(u * kUnitSegs, a.M, a.L), ue = seg_begin(useg1, a.M, a.L);

  // destination of this unit
  AT* dst = out;
  uint32_t lo = 0;
  bool use_smem = false;
  if constexpr (POL == kSmem) {
    if (warp == 0) {
      const int64_t seg = u * kUnitSegs + lane;
      uint32_t l0 = 0xffffffffu, h0 = 0;
      if (lane < kUnitSegs && seg < a.L) {
        const int Nm = a.dp.nmodes;
        const uint32_t s0 = a.ivl[(seg * Nm + a.out_mode) * 2], e0 = a.ivl[(seg * Nm + a.out_mode) * 2 + 1];
        if (e0 >= s0) {
          l0 = s0;
          h0 = e0;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        l0 = min(l0, __shfl_xor_sync(0xffffffffu, l0, o));
        h0 = max(h0, __shfl_xor_sync(0xffffffffu, h0, o));
      }
      if (lane == 0) {
        s_lorows[0] = l0;
        s_lorows[1] = (h0 >= l0) ? h0 - l0 + 1 : 0;
      }
    }
    __syncthreads();
    lo = s_lorows[0];
    const uint32_t rows = s_lorows[1];
    use_smem = rows <= static_cast<uint32_t>(a.smem_rows);
    if (use_smem) {
      AT* temp = reinterpret_cast<AT*>(dyn);
      uint32_t* touched = reinterpret_cast<uint32_t*>(temp + static_cast<size_t>(a.smem_rows) * R);
      for (uint32_t i = threadIdx.x; i < rows * R; i += kThreads) temp[i] = AT(0);
      for (uint32_t i = threadIdx.x; i < (rows + 31) / 32; i += kThreads) touched[i] = 0;
      dst = temp;
    }
    __syncthreads();
  } else if constexpr (POL == kTemp) {
    dst = static_cast<AT*>(a.temp) + a.toff[u];
    lo = a.ulo[u];
  }

  // chunks of this unit: warp w takes w, w + 8, ...
  int64_t base = ub + static_cast<int64_t>(warp) * 32;
  CKey<W32> kn{};
  typename VRaw<VT>::T vn{};
  if (base + lane < ue) {
    kn = load_ckey<W32>(a.keys, base + lane);
    vn = load_value_raw<VT>(a, base + lane);
  }
  for (; base < ue; base += kWarps * 32) {
    const int cnt = static_cast<int>(ue - base < 32 ? ue - base : 32);
    const bool ok = lane < cnt;
    const CKey<W32> k = kn;
    const typename VRaw<VT>::T vraw = vn;
    const int64_t nb = base + kWarps * 32;
    if (nb + lane < ue) {  // prefetch the warp's next chunk
      kn = load_ckey<W32>(a.keys, nb + lane);
      vn = load_value_raw<VT>(a, nb + lane);
    }
    const VT v = value_of<VT>(a, vraw, base + lane);
    uint32_t id[N];
#pragma unroll
    for (int s = 0; s < N; ++s) id[s] = extract_c<W32>(k, a.dp, s);
    if constexpr (POL == kWarpAgg) {
      // hot rows are staged as (bit 31 | table slot); the host enables the
      // table only when every output row is below 2^31.  Only nonzeros
      // whose key carries the hot-row flag probe the table.
      if (H > 0 && ok && (a.hot_key_bit < 0 || ckey_bit<W32>(k, a.hot_key_bit))) {
        const int slot = hot_lookup(st.hkeys, st.hidx, id[N - 1], a.hot_bits);
        if (slot >= 0) id[N - 1] = 0x80000000u | static_cast<uint32_t>(slot);
      }
    }
    int pos = lane;
    if constexpr (AGG) {
      const unsigned long long tag = ok ? static_cast<unsigned long long>(id[N - 1]) : (0x100000000ull + lane);
      const uint32_t peers = __match_any_sync(0xffffffffu, tag);
      const int leader = __ffs(peers) - 1;
      const uint32_t sz = (lane == leader) ? __popc(peers) : 0u;
      uint32_t inc = sz;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t start = __shfl_sync(0xffffffffu, inc - sz, leader);
      pos = static_cast<int>(start + __popc(peers & lt));
    }
    if (ok) stage_store<N, VT>(s_stage[warp][pos], id, v);
    __syncwarp();

    // group g: positions g*PER .. g*PER + PER - 1, with the gathers of the
    // next kGatherDepth positions in flight.  Loads past the chunk's end read
    // its last valid slot again (harmless, the result is not used), so every
    // load is unconditional and the pipeline registers rename instead of
    // being copied.
    const int p0 = g * PER;
    constexpr int D = PER < kGatherDepth ? PER : kGatherDepth;
    Pos<N, VT> q[D + 1];        // q[0]: the position being summed; q[1..D]: gathers in flight
    Rows<N, R, FT> rw[D + 1];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const int p = p0 + i;
      q[i] = stage_load<N, VT>(s_stage[warp][p < cnt ? p : cnt - 1]);
      gather<N, R, FT>(a, q[i], c, rw[i]);
    }
    AT acc[K];
#pragma unroll
    for (int e = 0; e < K; ++e) acc[e] = AT(0);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int p = p0 + j;
      const bool has = p < cnt;
      const bool hasn = (j + 1 < PER) && (p + 1 < cnt);
      if (j + D < PER) {
        const int pn = p + D;
        q[D] = stage_load<N, VT>(s_stage[warp][pn < cnt ? pn : cnt - 1]);
        gather<N, R, FT>(a, q[D], c, rw[D]);
      }
      const Pos<N, VT>& cur = q[0];
      if (has) {
        const uint32_t row = cur.id[N - 1];
        if constexpr (POL == kAtomic) {
          AT t[K];
          product<N, R, FT>(cur, rw[0], t);
          flush_global<R, FT>(out + static_cast<size_t>(row) * R, c, t);
        } else {
          accumulate<N, R, FT>(cur, rw[0], acc);
          if (!hasn || q[1].id[N - 1] != row) {
            if constexpr (POL == kSmem) {
              if (use_smem) {
                flush_shared<R, FT>(dst + static_cast<size_t>(row - lo) * R, c, acc);
                if (c == 0) {
                  uint32_t* touched = reinterpret_cast<uint32_t*>(reinterpret_cast<AT*>(dyn) +
                                                                  static_cast<size_t>(a.smem_rows) * R);
                  atomicOr(touched + ((row - lo) >> 5), 1u << ((row - lo) & 31));
                }
              } else {
                flush_global<R, FT>(out + static_cast<size_t>(row) * R, c, acc);
              }
            } else if constexpr (POL == kWarpAgg) {
              if (row & 0x80000000u)
                flush_global<R, FT>(st.hdata + static_cast<size_t>(row & 0x7fffffffu) * R, c, acc);
              else
                flush_global<R, FT>(out + static_cast<size_t>(row) * R, c, acc);
            } else {
              flush_global<R, FT>(dst + static_cast<size_t>(row - lo) * R, c, acc);
            }
#pragma unroll
            for (int e = 0; e < K; ++e) acc[e] = AT(0);
          }
        }
      }
      // advance the pipeline (register renames once unrolled)
#pragma unroll
      for (int i = 0; i < D; ++i) {
        q[i] = q[i + 1];
        rw[i] = rw[i + 1];
      }
    }
    __syncwarp();
  }

  if constexpr (POL == kSmem) {
    __syncthreads();
    if (use_smem) {
      const AT* temp = reinterpret_cast<const AT*>(dyn);
      const uint32_t* touched = reinterpret_cast<const uint32_t*>(temp + static_cast<size_t>(a.smem_rows) * R);
      const uint32_t rows = s_lorows[1];
      const int cc = threadIdx.x % LPN;
      for (uint32_t w = threadIdx.x / LPN; w < rows; w += kThreads / LPN) {
        if ((touched[w >> 5] >> (w & 31)) & 1u) {
          AT vals[K];
#pragma unroll
          for (int q = 0; q < C::PAIRS; ++q)
#pragma unroll
            for (int e = 0; e < C::VEC; ++e)
              vals[q * C::VEC + e] = temp[static_cast<size_t>(w) * R + cc * C::VEC + q * C::STRIDE + e];
          flush_global<R, FT>(out + static_cast<size_t>(lo + w) * R, cc, vals);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace alto

#include "mttkrp_fused.cuh"

namespace alto {

// One MTTKRP: persistent blocks stride over the units.
// FUSED selects the fused body (ATOMIC / WARPAGG only), which holds more
// gathers in flight and therefore runs fewer, larger-register blocks per SM.
#ifndef ALTO_FUSED_BLOCKS
#define ALTO_FUSED_BLOCKS 2
#endif
constexpr int kFusedBlocks = ALTO_FUSED_BLOCKS;

template <int N, int W32, int R, typename FT, int POL, bool FUSED = false>
__global__ void __launch_bounds__(kThreads, FUSED ? kFusedBlocks : 4) mttkrp_kernel(const __grid_constant__ MttkrpArgs a) {
  using AT = typename FTraits<FT>::AT;
  using VT = typename FTraits<FT>::VT;
  __shared__ uint4 s_stage[kWarps][32][Stage<N, VT>::W4];
  __shared__ uint32_t s_lorows[2];
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ uint4 s_stage2[FUSED ? 2 : 1][kWarps][32][Stage<N, VT>::W4];
  BlockState<AT> st{0, nullptr, nullptr, nullptr};
  if constexpr (POL == kWarpAgg) st = hot_table<AT, R>(a, dyn, blockIdx.x % kHotReplicas);
  const int64_t units = (a.L + kUnitSegs - 1) / kUnitSegs;
  if constexpr (FUSED && (POL == kAtomic || POL == kWarpAgg)) {
    process_units_fused<N, W32, R, FT, POL>(a, blockIdx.x, gridDim.x, units, st, s_stage2);
  } else {
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x)
      process_unit<N, W32, R, FT, POL>(a, u, st, s_stage, s_lorows, dyn);
  }
}

// Many MTTKRPs of one kernel shape in one persistent launch (the batched
// entry point): items[i] describes MTTKRP i, unit_prefix[i] its first global
// unit.  Each block takes a contiguous range of global units, so it switches
// items rarely; on a switch it copies the item's description to shared
// memory and rebuilds its hot-row table.
struct BatchArgs {
  const MttkrpArgs* items;
  const int64_t* unit_prefix;  // nitems + 1
  int nitems;
  int hot_replicas;            // copies of each item's hot rows
};

template <int N, int W32, int R, typename FT, int POL, bool FUSED = false>
__global__ void __launch_bounds__(kThreads, FUSED ? kFusedBlocks : 4) mttkrp_batch_kernel(const __grid_constant__ BatchArgs b) {
  using AT = typename FTraits<FT>::AT;
  using VT = typename FTraits<FT>::VT;
  __shared__ uint4 s_stage[kWarps][32][Stage<N, VT>::W4];
  __shared__ uint32_t s_lorows[2];
  __shared__ __align__(16) MttkrpArgs s_args;
  __shared__ uint4 s_stage2[FUSED ? 2 : 1][kWarps][32][Stage<N, VT>::W4];
  extern __shared__ __align__(16) unsigned char dyn[];
  const int64_t total = b.unit_prefix[b.nitems];
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t g0 = static_cast<int64_t>(blockIdx.x) * per;
  const int64_t g1 = g0 + per < total ? g0 + per : total;
  if (g0 >= g1) return;
  // item of the first unit: binary search over the prefix
  int lo = 0, hi = b.nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.unit_prefix[mid] <= g0) lo = mid; else hi = mid - 1;
  }
  int item = -1;
  BlockState<AT> st{0, nullptr, nullptr, nullptr};
  for (int64_t gu = g0; gu < g1; ++gu) {
    int want = item < 0 ? lo : item;
    while (gu >= b.unit_prefix[want + 1]) ++want;
    if (want != item) {
      item = want;
      __syncthreads();
      const uint32_t* src = reinterpret_cast<const uint32_t*>(b.items + item);
      uint32_t* d = reinterpret_cast<uint32_t*>(&s_args);
      for (int i = threadIdx.x; i < static_cast<int>(sizeof(MttkrpArgs) / 4); i += kThreads) d[i] = src[i];
      __syncthreads();
      if constexpr (POL == kWarpAgg) st = hot_table<AT, R>(s_args, dyn, blockIdx.x % b.hot_replicas);
    }
    if constexpr (FUSED && (POL == kAtomic || POL == kWarpAgg))
      process_units_fused<N, W32, R, FT, POL>(s_args, gu - b.unit_prefix[item], 1, gu - b.unit_prefix[item] + 1,
                                              st, s_stage2);
    else
      process_unit<N, W32, R, FT, POL>(s_args, gu - b.unit_prefix[item], st, s_stage, s_lorows, dyn);
  }
}

// out[hot[h], :] = sum over the replicas of rep[k, h, :] (every contribution
// to a row in the hot table went to the replicas, none to the output)
template <typename AT>
__global__ void __launch_bounds__(256) hot_reduce_kernel(const AT* __restrict__ rep, const uint32_t* __restrict__ hot,
                                                         int H, int R, int nrep, AT* __restrict__ out) {
  const int total = H * R;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    AT s = AT(0);
    for (int k = 0; k < nrep; ++k) s += rep[static_cast<size_t>(k) * total + e];
    const int h = e / R, r = e - h * R;
    out[static_cast<size_t>(hot[h]) * R + r] = s;
  }
}

// The same for many MTTKRPs at once: item i owns elements
// [prefix[i], prefix[i+1]) of the flattened (row, column) space.
struct HotItem {
  const void* rep;
  const uint32_t* hot;
  void* out;
  int H;
  int R;
  int nrep;
  int pad;
};

template <typename AT>
__global__ void __launch_bounds__(256) hot_reduce_batch_kernel(const HotItem* __restrict__ items,
                                                               const int64_t* __restrict__ prefix, int n) {
  const int64_t total = prefix[n];
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const HotItem it = items[lo];
    const int64_t q = e - prefix[lo];
    const int64_t tot = static_cast<int64_t>(it.H) * it.R;
    const AT* rep = static_cast<const AT*>(it.rep);
    AT s = AT(0);
    for (int k = 0; k < it.nrep; ++k) s += rep[k * tot + q];
    const int64_t h = q / it.R, r = q - h * it.R;
    static_cast<AT*>(it.out)[static_cast<size_t>(it.hot[h]) * it.R + r] = s;
  }
}

// Any order (runtime N <= kMaxModes) and any rank: one warp per segment,
// lanes stride over the rank, scalar atomics.
template <int W32, typename FT>
__global__ void __launch_bounds__(kThreads) mttkrp_generic_kernel(const __grid_constant__ MttkrpArgs a) {
  using AT = typename FTraits<FT>::AT;
  using VT = typename FTraits<FT>::VT;
  __shared__ uint32_t s_idx[kWarps][kMaxModes][32];
  __shared__ VT s_val[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Nm = a.dp.nmodes, R = a.R;
  AT* out = static_cast<AT*>(a.out);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kWarps;
  for (int64_t seg = static_cast<int64_t>(blockIdx.x) * kWarps + warp; seg < a.L; seg += nw) {
    const int64_t s0 = seg_begin(seg, a.M, a.L), s1 = seg_begin(seg + 1, a.M, a.L);
    for (int64_t base = s0; base < s1; base += 32) {
      const int cnt = static_cast<int>(s1 - base < 32 ? s1 - base : 32);
      if (lane < cnt) {
        const CKey<W32> k = load_ckey<W32>(a.keys, base + lane);
        for (int s = 0; s < Nm; ++s) s_idx[warp][s][lane] = extract_c<W32>(k, a.dp, s);
        s_val[warp][lane] = load_value<VT>(a, base + lane);
      }
      __syncwarp();
      for (int p = 0; p < cnt; ++p) {
        const uint32_t row = s_idx[warp][Nm - 1][p];
        for (int r = lane; r < R; r += 32) {
          AT t = static_cast<AT>(s_val[warp][p]);
          for (int s = 0; s < Nm - 1; ++s) {
            const FT* f = static_cast<const FT*>(a.f[s]);
            t *= static_cast<AT>(f[static_cast<size_t>(s_idx[warp][s][p]) * R + r]);
          }
          atomicAdd(out + static_cast<size_t>(row) * R + r, t);
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// launch description shared by the per-dtype dispatchers
struct MttkrpLaunch {
  MttkrpArgs args;
  int N;
  int W32;
  int variant;   // ATOMIC / WARPAGG / SMEM / TEMP (the generic kernel ignores it)
  int sms;       // SM count of the device
  size_t smem_dyn;
  bool fused;    // ATOMIC / WARPAGG through the fused body
  bool generic;  // the rank- and order-generic kernel whatever the shape
};

// per factor type and stored key width (W32 32-bit words), one translation unit each
#define ALTO_DECLARE_DISPATCH(T, WW)                                                        \
  cudaError_t mttkrp_dispatch_##T##_w##WW(const MttkrpLaunch& l, cudaStream_t s);           \
  cudaError_t mttkrp_batch_dispatch_##T##_w##WW(const struct BatchLaunch& l, cudaStream_t s);
ALTO_DECLARE_DISPATCH(f32, 1)
ALTO_DECLARE_DISPATCH(f32, 2)
ALTO_DECLARE_DISPATCH(f32, 3)
ALTO_DECLARE_DISPATCH(f32, 4)
ALTO_DECLARE_DISPATCH(f64, 1)
ALTO_DECLARE_DISPATCH(f64, 2)
ALTO_DECLARE_DISPATCH(f64, 3)
ALTO_DECLARE_DISPATCH(f64, 4)
ALTO_DECLARE_DISPATCH(bf16, 1)
ALTO_DECLARE_DISPATCH(bf16, 2)
ALTO_DECLARE_DISPATCH(bf16, 3)
ALTO_DECLARE_DISPATCH(bf16, 4)
#undef ALTO_DECLARE_DISPATCH

// launch description of one group of the batched entry point
struct BatchLaunch {
  BatchArgs args;
  int N;
  int W32;
  int R;
  int variant;   // ATOMIC / WARPAGG / SMEM
  int sms;
  size_t smem_dyn;
  int64_t units;  // thread-block units of all items
  bool fused;     // ATOMIC / WARPAGG through the fused body
};

#define ALTO_PICK_W(T, KIND, L, S)                                     \
  switch ((L).W32) {                                                   \
    case 1: return mttkrp_##KIND##dispatch_##T##_w1(L, S);             \
    case 2: return mttkrp_##KIND##dispatch_##T##_w2(L, S);             \
    case 3: return mttkrp_##KIND##dispatch_##T##_w3(L, S);             \
    default: return mttkrp_##KIND##dispatch_##T##_w4(L, S);            \
  }

inline cudaError_t mttkrp_batch_dispatch(const BatchLaunch& l, alto_dtype fdtype, cudaStream_t s) {
  switch (fdtype) {
    case ALTO_F64: ALTO_PICK_W(f64, batch_, l, s)
    case ALTO_F32: ALTO_PICK_W(f32, batch_, l, s)
    default: ALTO_PICK_W(bf16, batch_, l, s)
  }
}

template <typename Kern>
cudaError_t launch_batch(Kern kern, const BatchLaunch& l, cudaStream_t s) {
  // the default dynamic limit is 48 KB minus the kernel's static shared
  // memory: raise it for every launch that uses dynamic shared memory
  if (l.smem_dyn > 0) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(l.smem_dyn));
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, l.smem_dyn);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  // every group may fill the device; groups on parallel graph branches take
  // over the SMs that earlier groups' blocks release
  int64_t g = static_cast<int64_t>(l.sms) * occ;
  if (g > l.units) g = l.units;
  if (g < 1) g = 1;
  kern<<<static_cast<unsigned>(g), kThreads, l.smem_dyn, s>>>(l.args);
  note_launch();
  return cudaGetLastError();
}

template <typename FT, int W32>
cudaError_t mttkrp_batch_dispatch_typed(const BatchLaunch& l, cudaStream_t s) {
#define ALTO_BLAUNCH_NR(NN, RR)                                                                  \
  do {                                                                                           \
    switch (l.variant) {                                                                         \
      case kSmem: return launch_batch(mttkrp_batch_kernel<NN, W32, RR, FT, kSmem>, l, s);          \
      case kAtomic:                                                                              \
        if (l.fused) return launch_batch(mttkrp_batch_kernel<NN, W32, RR, FT, kAtomic, true>, l, s); \
        return launch_batch(mttkrp_batch_kernel<NN, W32, RR, FT, kAtomic>, l, s);                  \
      default:                                                                                   \
        if (l.fused) return launch_batch(mttkrp_batch_kernel<NN, W32, RR, FT, kWarpAgg, true>, l, s); \
        return launch_batch(mttkrp_batch_kernel<NN, W32, RR, FT, kWarpAgg>, l, s);                 \
    }                                                                                            \
  } while (0)
#define ALTO_BLAUNCH_R(NN)              \
  do {                                  \
    switch (l.R) {                      \
      case 8: ALTO_BLAUNCH_NR(NN, 8);   \
      case 16: ALTO_BLAUNCH_NR(NN, 16); \
      case 32: ALTO_BLAUNCH_NR(NN, 32); \
      case 64: ALTO_BLAUNCH_NR(NN, 64); \
      default: break;                   \
    }                                   \
  } while (0)
  switch (l.N) {
    case 2: ALTO_BLAUNCH_R(2); break;
    case 3: ALTO_BLAUNCH_R(3); break;
    case 4: ALTO_BLAUNCH_R(4); break;
    case 5: ALTO_BLAUNCH_R(5); break;
    default: break;
  }
#undef ALTO_BLAUNCH_R
#undef ALTO_BLAUNCH_NR
  return cudaErrorInvalidValue;  // the host only groups specialised shapes
}

inline cudaError_t mttkrp_dispatch(const MttkrpLaunch& l, alto_dtype fdtype, cudaStream_t s) {
  switch (fdtype) {
    case ALTO_F64: ALTO_PICK_W(f64, , l, s)
    case ALTO_F32: ALTO_PICK_W(f32, , l, s)
    default: ALTO_PICK_W(bf16, , l, s)
  }
}

// Persistent launch: as many blocks as fit on the device at once (never more
// than the work units), each striding over the units.
template <typename Kern>
cudaError_t launch_persistent(Kern kern, const MttkrpLaunch& l, size_t smem, int64_t units, cudaStream_t s) {
  if (smem > 0) {  // the default limit is 48 KB minus the static shared memory
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  int64_t g = static_cast<int64_t>(l.sms) * occ;
  if (g > units) g = units;
  if (g < 1) g = 1;
  kern<<<static_cast<unsigned>(g), kThreads, smem, s>>>(l.args);
  note_launch();
  return cudaGetLastError();
}

// Instantiate and launch for one factor type and key width.
template <typename FT, int W32>
cudaError_t mttkrp_dispatch_typed(const MttkrpLaunch& l, cudaStream_t s) {
  const MttkrpArgs& a = l.args;
  const int64_t units = (a.L + kUnitSegs - 1) / kUnitSegs;
  if (l.generic) return launch_persistent(mttkrp_generic_kernel<W32, FT>, l, 0, (a.L + kWarps - 1) / kWarps, s);
#define ALTO_LAUNCH_NR(NN, RR)                                                                           \
  do {                                                                                                   \
    switch (l.variant) {                                                                                 \
      case kSmem: return launch_persistent(mttkrp_kernel<NN, W32, RR, FT, kSmem>, l, l.smem_dyn, units, s); \
      case kTemp: return launch_persistent(mttkrp_kernel<NN, W32, RR, FT, kTemp>, l, 0, units, s);        \
      case kWarpAgg:                                                                                     \
        if (l.fused) return launch_persistent(mttkrp_kernel<NN, W32, RR, FT, kWarpAgg, true>, l, l.smem_dyn, units, s); \
        return launch_persistent(mttkrp_kernel<NN, W32, RR, FT, kWarpAgg>, l, l.smem_dyn, units, s);    \
      default:                                                                                           \
        if (l.fused) return launch_persistent(mttkrp_kernel<NN, W32, RR, FT, kAtomic, true>, l, 0, units, s); \
        return launch_persistent(mttkrp_kernel<NN, W32, RR, FT, kAtomic>, l, 0, units, s);              \
    }                                                                                                    \
  } while (0)
#define ALTO_LAUNCH_R(NN)              \
  do {                                 \
    switch (a.R) {                     \
      case 8: ALTO_LAUNCH_NR(NN, 8);   \
      case 16: ALTO_LAUNCH_NR(NN, 16); \
      case 32: ALTO_LAUNCH_NR(NN, 32); \
      case 64: ALTO_LAUNCH_NR(NN, 64); \
      default: break;                  \
    }                                  \
  } while (0)
  switch (l.N) {
    case 2: ALTO_LAUNCH_R(2); break;
    case 3: ALTO_LAUNCH_R(3); break;
    case 4: ALTO_LAUNCH_R(4); break;
    case 5: ALTO_LAUNCH_R(5); break;
    default: break;
  }
#undef ALTO_LAUNCH_R
#undef ALTO_LAUNCH_NR
  return launch_persistent(mttkrp_generic_kernel<W32, FT>, l, 0, (a.L + kWarps - 1) / kWarps, s);
}

// Whether the specialised kernels cover (N, R); otherwise the generic one runs.
inline bool mttkrp_specialised(int N, int R) {
  return N >= 2 && N <= 5 && (R == 8 || R == 16 || R == 32 || R == 64);
}

}  // namespace alto
