// MTTKRP over the ALTO format (Sec. 2.2, Alg. 1-2), GPU kernel family.
//
// Work split: the ordered nonzeros are cut into L equal-nnz line segments
// (Sec. 3.2).  Every segment is processed by one warp, 32 nonzeros at a
// time:
//   1. each lane streams one key and value and de-linearizes all N indices
//      (bit-level compress, EXTRACT of Alg. 2);
//   2. the decoded tuples are staged in shared memory;
//   3. lanes form groups of R/VEC lanes, a group owning one nonzero at a
//      time and VEC consecutive columns per lane; each lane gathers its VEC
//      columns of the N-1 input factor rows, multiplies them with the value
//      (Hadamard product of Alg. 2) and accumulates into the output row.
//
// Output accumulation variants (Alg. 2 and the Sec. 3.3 rule):
//   ATOMIC  every nonzero issues a vector atomic into the output row (the
//           ATOMIC branch of Alg. 2);
//   WARPAGG the 32 staged nonzeros are reordered by output row inside the
//           warp (match on the row, prefix over the matched sets) so that
//           equal rows are consecutive; a group sums its run of an equal row
//           in registers and issues one atomic per run;
//   SMEM    a thread block takes 8 consecutive segments, sizes a Temp in
//           shared memory by their output-mode interval T (Alg. 2, Temp_l),
//           accumulates there with shared-memory atomics and then flushes
//           every touched row once into the output; a block whose interval
//           does not fit falls back to direct atomics.
// All variants compute the same sum; only the rounding order differs.
#pragma once

#include "internal.h"

namespace alto {

// ---------------------------------------------------------------------------
// factor element traits: 16-byte vector loads of VEC elements
template <typename FT>
struct FTraits;
template <>
struct FTraits<float> {
  static constexpr int VEC = 4;
  using AT = float;
};
template <>
struct FTraits<double> {
  static constexpr int VEC = 2;
  using AT = double;
};
template <>
struct FTraits<__nv_bfloat16> {
  static constexpr int VEC = 8;
  using AT = float;
};

template <typename FT>
__device__ __forceinline__ void load_vec(const FT* p, typename FTraits<FT>::AT* v);

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
__device__ __forceinline__ void load_vec<__nv_bfloat16>(const __nv_bfloat16* p, float* v) {
  const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __nv_bfloat162 h;
    memcpy(&h, &w[j], 4);
    const float2 f = __bfloat1622float2(h);
    v[2 * j] = f.x;
    v[2 * j + 1] = f.y;
  }
}

// vector atomic add of VEC accumulators into out (FP32 or FP64)
template <int VEC>
__device__ __forceinline__ void atomic_vec(float* out, const float* v) {
#pragma unroll
  for (int j = 0; j < VEC; j += 4) red_add_v4(out + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
}
template <int VEC>
__device__ __forceinline__ void atomic_vec(double* out, const double* v) {
#pragma unroll
  for (int j = 0; j < VEC; ++j) red_add_f64(out + j, v[j]);
}

template <typename AT>
__device__ __forceinline__ AT load_val(const void* vals, int64_t x) {
  return __ldcs(static_cast<const AT*>(vals) + x);
}

struct MttkrpArgs {
  const uint64_t* keys;
  const void* vals;   // FP64 when the factors are FP64, else FP32
  int64_t M;
  int64_t L;          // line segments
  const void* f[kMaxModes];  // factor of each decode slot; slot N-1 is the output mode
  void* out;
  int R;
  int out_mode;       // mode of the output (column of the interval table)
  const uint32_t* ivl;       // L x N x 2 segment intervals
  int smem_rows;      // SMEM variant: rows of the shared Temp
  DecodeParams dp;
};

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

// ---------------------------------------------------------------------------
// Decode one chunk of up to 32 nonzeros starting at `base` into shared
// staging.  With AGG the chunk is reordered so equal output rows are
// consecutive.  Returns the number of valid nonzeros.
template <int N, int KW, typename AT, bool AGG>
__device__ __forceinline__ int stage_chunk(const MttkrpArgs& a, int64_t base, int64_t end, int lane,
                                           uint32_t (*s_idx)[32], AT* s_val) {
  const int cnt = static_cast<int>(end - base < 32 ? end - base : 32);
  const bool ok = lane < cnt;
  uint32_t id[N];
  AT v = AT(0);
  if (ok) {
    const KeyT<KW> k = load_key<KW>(a.keys, base + lane);
#pragma unroll
    for (int s = 0; s < N; ++s) id[s] = extract<KW>(k, a.dp, s);
    v = load_val<AT>(a.vals, base + lane);
  }
  int pos = lane;
  if constexpr (AGG) {
    const unsigned long long tag =
        ok ? static_cast<unsigned long long>(id[N - 1]) : (0x100000000ull + lane);
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
    pos = static_cast<int>(start + __popc(peers & lanemask_lt()));
  }
  if (ok) {
#pragma unroll
    for (int s = 0; s < N; ++s) s_idx[s][pos] = id[s];
    s_val[pos] = v;
  }
  __syncwarp();
  return cnt;
}

// product v * prod_{s < N-1} U_s[i_s, cols] for one staged nonzero
template <int N, int R, typename FT>
__device__ __forceinline__ void nnz_product(const MttkrpArgs& a, const uint32_t (*s_idx)[32],
                                            const typename FTraits<FT>::AT* s_val, int p, int c,
                                            typename FTraits<FT>::AT* prod) {
  using AT = typename FTraits<FT>::AT;
  constexpr int VEC = FTraits<FT>::VEC;
  const AT v = s_val[p];
#pragma unroll
  for (int e = 0; e < VEC; ++e) prod[e] = v;
#pragma unroll
  for (int s = 0; s < N - 1; ++s) {
    const FT* row = static_cast<const FT*>(a.f[s]) + static_cast<size_t>(s_idx[s][p]) * R + c * VEC;
    AT u[VEC];
    load_vec<FT>(row, u);
#pragma unroll
    for (int e = 0; e < VEC; ++e) prod[e] *= u[e];
  }
}

// ATOMIC (AGG = false) and WARPAGG (AGG = true)
template <int N, int KW, int R, typename FT, bool AGG>
__global__ void __launch_bounds__(kThreads) mttkrp_warp_kernel(const __grid_constant__ MttkrpArgs a) {
  using AT = typename FTraits<FT>::AT;
  constexpr int VEC = FTraits<FT>::VEC;
  constexpr int LPN = R / VEC;       // lanes per nonzero
  constexpr int PER = LPN;           // staged positions per group (32 / groups)
  static_assert(LPN >= 1 && LPN <= 32 && 32 % LPN == 0, "rank / vector width");
  __shared__ uint32_t s_idx[kWarps][N][32];
  __shared__ AT s_val[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / LPN, c = lane % LPN;
  AT* out = static_cast<AT*>(a.out);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kWarps;
  for (int64_t seg = static_cast<int64_t>(blockIdx.x) * kWarps + warp; seg < a.L; seg += nw) {
    const int64_t s0 = seg_begin(seg, a.M, a.L), s1 = seg_begin(seg + 1, a.M, a.L);
    for (int64_t base = s0; base < s1; base += 32) {
      const int cnt = stage_chunk<N, KW, AT, AGG>(a, base, s1, lane, s_idx[warp], s_val[warp]);
      AT acc[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = AT(0);
#pragma unroll 2
      for (int j = 0; j < PER; ++j) {
        const int p = g * PER + j;
        if (p >= cnt) break;
        const uint32_t row = s_idx[warp][N - 1][p];
        AT prod[VEC];
        nnz_product<N, R, FT>(a, s_idx[warp], s_val[warp], p, c, prod);
        if constexpr (AGG) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[e] += prod[e];
          const bool last = (j == PER - 1) || (p + 1 >= cnt) || (s_idx[warp][N - 1][p + 1] != row);
          if (last) {
            atomic_vec<VEC>(out + static_cast<size_t>(row) * R + c * VEC, acc);
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[e] = AT(0);
          }
        } else {
          atomic_vec<VEC>(out + static_cast<size_t>(row) * R + c * VEC, prod);
        }
      }
      __syncwarp();
    }
  }
}

// SMEM: 8 segments per block, Temp in shared memory over the union of their
// output-mode intervals; direct atomics when the interval is too wide.
template <int N, int KW, int R, typename FT>
__global__ void __launch_bounds__(kThreads) mttkrp_smem_kernel(const __grid_constant__ MttkrpArgs a) {
  using AT = typename FTraits<FT>::AT;
  constexpr int VEC = FTraits<FT>::VEC;
  constexpr int LPN = R / VEC;
  constexpr int PER = LPN;
  __shared__ uint32_t s_idx[kWarps][N][32];
  __shared__ AT s_val[kWarps][32];
  __shared__ uint32_t s_lo, s_rows;
  extern __shared__ __align__(16) unsigned char dyn[];
  AT* temp = reinterpret_cast<AT*>(dyn);
  uint32_t* touched = reinterpret_cast<uint32_t*>(temp + static_cast<size_t>(a.smem_rows) * R);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / LPN, c = lane % LPN;
  AT* out = static_cast<AT*>(a.out);
  const int64_t units = (a.L + kWarps - 1) / kWarps;
  const int Nm = a.dp.nmodes;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    if (warp == 0) {
      const int64_t seg = u * kWarps + lane;
      uint32_t lo = 0xffffffffu, hi = 0;
      if (lane < kWarps && seg < a.L) {
        const uint32_t s = a.ivl[(seg * Nm + a.out_mode) * 2], e = a.ivl[(seg * Nm + a.out_mode) * 2 + 1];
        if (e >= s) {
          lo = s;
          hi = e;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) {
        s_lo = lo;
        s_rows = (hi >= lo) ? hi - lo + 1 : 0;
      }
    }
    __syncthreads();
    const uint32_t lo = s_lo, rows = s_rows;
    const bool fits = rows <= static_cast<uint32_t>(a.smem_rows);
    if (fits) {
      for (uint32_t i = threadIdx.x; i < rows * R; i += kThreads) temp[i] = AT(0);
      for (uint32_t i = threadIdx.x; i < (rows + 31) / 32; i += kThreads) touched[i] = 0;
    }
    __syncthreads();
    const int64_t seg = u * kWarps + warp;
    if (seg < a.L) {
      const int64_t s0 = seg_begin(seg, a.M, a.L), s1 = seg_begin(seg + 1, a.M, a.L);
      for (int64_t base = s0; base < s1; base += 32) {
        const int cnt = stage_chunk<N, KW, AT, false>(a, base, s1, lane, s_idx[warp], s_val[warp]);
#pragma unroll 2
        for (int j = 0; j < PER; ++j) {
          const int p = g * PER + j;
          if (p >= cnt) break;
          const uint32_t row = s_idx[warp][N - 1][p];
          AT prod[VEC];
          nnz_product<N, R, FT>(a, s_idx[warp], s_val[warp], p, c, prod);
          if (fits) {
            AT* t = temp + static_cast<size_t>(row - lo) * R + c * VEC;
#pragma unroll
            for (int e = 0; e < VEC; ++e) atomicAdd(t + e, prod[e]);
            if (c == 0) atomicOr(touched + ((row - lo) >> 5), 1u << ((row - lo) & 31));
          } else {
            atomic_vec<VEC>(out + static_cast<size_t>(row) * R + c * VEC, prod);
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (fits) {
      // flush: one vector atomic per (touched row, lane slot)
      for (uint32_t w = threadIdx.x / LPN; w < rows; w += kThreads / LPN) {
        if ((touched[w >> 5] >> (w & 31)) & 1u) {
          const int cc = threadIdx.x % LPN;
          atomic_vec<VEC>(out + static_cast<size_t>(lo + w) * R + cc * VEC,
                          temp + static_cast<size_t>(w) * R + cc * VEC);
        }
      }
    }
    __syncthreads();
  }
}

// Any order (runtime N <= kMaxModes) and any rank: one warp per segment,
// lanes stride over the rank, scalar atomics.
template <int KW, typename FT>
__global__ void __launch_bounds__(kThreads) mttkrp_generic_kernel(const __grid_constant__ MttkrpArgs a) {
  using AT = typename FTraits<FT>::AT;
  __shared__ uint32_t s_idx[kWarps][kMaxModes][32];
  __shared__ AT s_val[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Nm = a.dp.nmodes, R = a.R;
  AT* out = static_cast<AT*>(a.out);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kWarps;
  for (int64_t seg = static_cast<int64_t>(blockIdx.x) * kWarps + warp; seg < a.L; seg += nw) {
    const int64_t s0 = seg_begin(seg, a.M, a.L), s1 = seg_begin(seg + 1, a.M, a.L);
    for (int64_t base = s0; base < s1; base += 32) {
      const int cnt = static_cast<int>(s1 - base < 32 ? s1 - base : 32);
      if (lane < cnt) {
        const KeyT<KW> k = load_key<KW>(a.keys, base + lane);
        for (int s = 0; s < Nm; ++s) s_idx[warp][s][lane] = extract<KW>(k, a.dp, s);
        s_val[warp][lane] = load_val<AT>(a.vals, base + lane);
      }
      __syncwarp();
      for (int p = 0; p < cnt; ++p) {
        const uint32_t row = s_idx[warp][Nm - 1][p];
        for (int r = lane; r < R; r += 32) {
          AT t = s_val[warp][p];
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
  int KW;
  int variant;   // ALTO_VAR_ATOMIC / WARPAGG / SMEM (the generic kernel ignores it)
  int sms;       // SM count of the device
  size_t smem_dyn;
};

cudaError_t mttkrp_dispatch_f32(const MttkrpLaunch& l, cudaStream_t s);
cudaError_t mttkrp_dispatch_f64(const MttkrpLaunch& l, cudaStream_t s);
cudaError_t mttkrp_dispatch_bf16(const MttkrpLaunch& l, cudaStream_t s);

// Persistent launch: as many blocks as fit on the device at once (never more
// than the work units), each striding over the units.
template <typename Kern>
cudaError_t launch_persistent(Kern kern, const MttkrpLaunch& l, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  const int64_t units = (l.args.L + kWarps - 1) / kWarps;
  int64_t g = static_cast<int64_t>(l.sms) * occ;
  if (g > units) g = units;
  if (g < 1) g = 1;
  kern<<<static_cast<unsigned>(g), kThreads, smem, s>>>(l.args);
  note_launch();
  return cudaGetLastError();
}

// Instantiate and launch for one factor type.
template <typename FT>
cudaError_t mttkrp_dispatch(const MttkrpLaunch& l, cudaStream_t s) {
  const MttkrpArgs& a = l.args;
#define ALTO_LAUNCH_NR(NN, KK, RR)                                                           \
  do {                                                                                      \
    if (l.variant == ALTO_VAR_SMEM)                                                         \
      return launch_persistent(mttkrp_smem_kernel<NN, KK, RR, FT>, l, l.smem_dyn, s);       \
    if (l.variant == ALTO_VAR_WARPAGG)                                                      \
      return launch_persistent(mttkrp_warp_kernel<NN, KK, RR, FT, true>, l, 0, s);          \
    return launch_persistent(mttkrp_warp_kernel<NN, KK, RR, FT, false>, l, 0, s);           \
  } while (0)
#define ALTO_LAUNCH_R(NN, KK)              \
  do {                                     \
    switch (a.R) {                         \
      case 8: ALTO_LAUNCH_NR(NN, KK, 8);   \
      case 16: ALTO_LAUNCH_NR(NN, KK, 16); \
      case 32: ALTO_LAUNCH_NR(NN, KK, 32); \
      case 64: ALTO_LAUNCH_NR(NN, KK, 64); \
      default: break;                      \
    }                                      \
  } while (0)
#define ALTO_LAUNCH_N(KK)           \
  do {                              \
    switch (l.N) {                  \
      case 2: ALTO_LAUNCH_R(2, KK); \
        break;                      \
      case 3: ALTO_LAUNCH_R(3, KK); \
        break;                      \
      case 4: ALTO_LAUNCH_R(4, KK); \
        break;                      \
      case 5: ALTO_LAUNCH_R(5, KK); \
        break;                      \
      default: break;               \
    }                               \
  } while (0)
  if (l.KW == 1) {
    ALTO_LAUNCH_N(1);
    return launch_persistent(mttkrp_generic_kernel<1, FT>, l, 0, s);
  }
  ALTO_LAUNCH_N(2);
  return launch_persistent(mttkrp_generic_kernel<2, FT>, l, 0, s);
#undef ALTO_LAUNCH_N
#undef ALTO_LAUNCH_R
#undef ALTO_LAUNCH_NR
}

// Whether the specialised kernels cover (N, R); otherwise the generic one runs.
inline bool mttkrp_specialised(int N, int R) {
  return N >= 2 && N <= 5 && (R == 8 || R == 16 || R == 32 || R == 64);
}

}  // namespace alto
