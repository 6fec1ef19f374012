// ALTO generation kernels other than the sort (Sec. 3.1-3.3):
//   encode         linearization: bit-level gather of every mode index into
//                  one key (Sec. 3.1);
//   permute        values into ALTO order;
//   sumsq          ||X||^2 for the CP-ALS fit (duplicates summed first);
//   segment_stats  per-segment mode intervals T_{l,n} (Sec. 3.2), plus the
//                  first and last segment touching every row, from which the
//                  distinct-row counts and the helper flags follow;
//   set_flags      boundary/internal helper flags in the spare key bits
//                  (Sec. 3.3).
#include "internal.h"

namespace alto {

namespace {

struct EncodeParams {
  int nmodes;
  uint64_t dims[kMaxModes];
  int nbits[kMaxModes];
};

// Bit-level deposit of every mode index into its key positions: per 32-bit
// key word, the slice of the index that the word holds is spread over the
// word's mask with the five-step parallel-suffix "expand" (Hacker's Delight,
// 2nd ed., Sec. 7-5), the inverse of the compress the kernels use to
// de-linearize, driven by the same move masks.
template <typename IT, int KW>
__global__ void __launch_bounds__(256) encode_kernel(const __grid_constant__ DecodeParams dp,
                                                     const __grid_constant__ EncodeParams ep,
                                                     const __grid_constant__ IdxPtrs idx, int64_t M,
                                                     uint64_t* __restrict__ keys, int* status) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < M; x += stride) {
    uint32_t w[2 * KW];
#pragma unroll
    for (int q = 0; q < 2 * KW; ++q) w[q] = 0;
    for (int n = 0; n < dp.nmodes; ++n) {
      uint64_t i = static_cast<uint64_t>(__ldcs(static_cast<const IT*>(idx.p[n]) + x));
      if (i >= ep.dims[n]) {
        set_status(status, ALTO_ERANGE);
        i = 0;
      }
      const uint32_t i32 = static_cast<uint32_t>(i);
#pragma unroll
      for (int q = 0; q < 2 * KW; ++q) {
        const uint32_t m = dp.mask[n][q];
        if (m != 0u) {
          uint32_t v = dp.shift[n][q] < 32 ? (i32 >> dp.shift[n][q]) : 0u;
#pragma unroll
          for (int k = 4; k >= 0; --k) {
            const uint32_t mv = dp.mv[n][q][k];
            v = (v & ~mv) | ((v << (1u << k)) & mv);
          }
          w[q] |= v & m;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < KW; ++q)
      keys[x * KW + q] = static_cast<uint64_t>(w[2 * q]) | (static_cast<uint64_t>(w[2 * q + 1]) << 32);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) permute_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                      const uint32_t* __restrict__ perm, int64_t M) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < M; x += stride)
    dst[x] = src[perm[x]];
}

__device__ __forceinline__ double value_f64(double v) { return v; }
__device__ __forceinline__ double value_f64(float v) { return static_cast<double>(v); }
__device__ __forceinline__ double value_f64(uint16_t b) {  // a BF16 value's bits
  return static_cast<double>(__uint_as_float(static_cast<uint32_t>(b) << 16));
}

// ||X||^2 where X sums duplicate coordinates: over the ordered keys, every
// run of equal keys contributes (sum of its values)^2.
template <typename T, int KW>
__global__ void __launch_bounds__(256) sumsq_kernel(const uint64_t* __restrict__ keys,
                                                    const T* __restrict__ v, int64_t M, double* out) {
  double s = 0.0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < M; x += stride) {
    bool start = x == 0;
    if (!start) {
#pragma unroll
      for (int w = 0; w < KW; ++w) start |= keys[x * KW + w] != keys[(x - 1) * KW + w];
    }
    if (!start) continue;
    double run = value_f64(v[x]);
    for (int64_t y = x + 1; y < M; ++y) {
      bool same = true;
#pragma unroll
      for (int w = 0; w < KW; ++w) same &= keys[y * KW + w] == keys[x * KW + w];
      if (!same) break;
      run += value_f64(v[y]);
    }
    s += run * run;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

struct RowArrays {
  uint32_t* first[kMaxModes];
  uint32_t* last[kMaxModes];
  uint32_t* cnt[kMaxModes];  // sampled nonzeros per row (every kHotSample-th)
};

// One warp per segment.  Lanes walk the segment 32 elements at a time,
// decode every mode, keep running min/max, and record the lowest / highest
// segment that touches each row and the sampled row counts.  Lanes holding
// the same row are matched first so that one lane per row issues the
// atomics, and a first/last value already at least as good is not touched:
// the heavy rows of skewed tensors would otherwise serialise on one address.
template <int KW>
__global__ void __launch_bounds__(256) segment_stats_kernel(const __grid_constant__ DecodeParams dp,
                                                            const uint64_t* __restrict__ keys,
                                                            int64_t M, int64_t L,
                                                            uint32_t* __restrict__ ivl,
                                                            const __grid_constant__ RowArrays ra) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int N = dp.nmodes;
  for (int64_t seg = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
       seg < L; seg += nwarps) {
    const int64_t s0 = seg_begin(seg, M, L), s1 = seg_begin(seg + 1, M, L);
    uint32_t lo[kMaxModes], hi[kMaxModes], prev[kMaxModes];
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n) {
      lo[n] = 0xffffffffu;
      hi[n] = 0;
      prev[n] = 0xffffffffu;
    }
    const uint32_t useg = static_cast<uint32_t>(seg);
    for (int64_t base = s0; base < s1; base += 32) {
      const int64_t x = base + lane;
      const bool ok = x < s1;
      KeyT<KW> k{};
      if (ok) k = load_key<KW>(keys, x);
      const uint32_t sampled = __ballot_sync(0xffffffffu, ok && (x % kHotSample) == 0);
#pragma unroll
      for (int n = 0; n < kMaxModes; ++n) {
        if (n < N) {
          const uint32_t i = extract<KW>(k, dp, n);
          if (ok) {
            lo[n] = min(lo[n], i);
            hi[n] = max(hi[n], i);
          }
          const unsigned long long tag = ok ? static_cast<unsigned long long>(i) : (0x100000000ull + lane);
          const uint32_t peers = __match_any_sync(0xffffffffu, tag);
          if (ok && lane == __ffs(peers) - 1 && i != prev[n]) {
            if (ra.first[n][i] > useg) atomicMin(ra.first[n] + i, useg);
            if (ra.last[n] != nullptr && ra.last[n][i] < useg) atomicMax(ra.last[n] + i, useg);
          }
          if (ok && lane == __ffs(peers) - 1) {
            prev[n] = i;
            const uint32_t ns = __popc(peers & sampled);
            if (ra.cnt[n] != nullptr && ns) atomicAdd(ra.cnt[n] + i, ns);
          }
        }
      }
    }
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n) {
      if (n < N) {
        uint32_t a = lo[n], b = hi[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
          b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
          if (s1 <= s0) {  // empty segment: (1, 0)
            a = 1;
            b = 0;
          }
          ivl[(seg * N + n) * 2 + 0] = a;
          ivl[(seg * N + n) * 2 + 1] = b;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256) count_touched_kernel(const uint32_t* __restrict__ first,
                                                            uint64_t n, unsigned long long* out) {
  unsigned long long c = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride)
    c += first[r] != 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void __launch_bounds__(256) max_interval_kernel(const uint32_t* __restrict__ ivl, int64_t L,
                                                           int N, unsigned long long* out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < L * N; j += stride) {
    const uint32_t a = ivl[2 * j], b = ivl[2 * j + 1];
    if (b >= a) atomicMax(out + (j % N), static_cast<unsigned long long>(b - a) + 1ull);
  }
}

struct FlagParams {
  int nflag;
  int slot[kMaxModes];  // decode slot (= mode) of each flagged mode
  int bit[kMaxModes];   // key bit of its flag
  int hot;              // 1: the flag marks a hot row (map lookup), 0: internal row
  const uint32_t* map[kMaxModes];  // hot: bitmap of the mode's hot rows
};

template <int KW>
__global__ void __launch_bounds__(256) set_flags_kernel(const __grid_constant__ DecodeParams dp,
                                                        const __grid_constant__ FlagParams fp,
                                                        uint64_t* __restrict__ keys, int64_t M,
                                                        const __grid_constant__ RowArrays ra) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < M; x += stride) {
    const KeyT<KW> k = load_key<KW>(keys, x);
    uint64_t w[2] = {0, 0};
    for (int f = 0; f < fp.nflag; ++f) {
      const int n = fp.slot[f];
      const uint32_t i = extract<KW>(k, dp, n);
      const bool set = fp.hot ? ((fp.map[f][i >> 5] >> (i & 31)) & 1u) != 0 : ra.first[n][i] == ra.last[n][i];
      if (set) w[fp.bit[f] >> 6] |= 1ull << (fp.bit[f] & 63);
    }
    keys[x * KW] |= w[0];
    if (KW == 2) keys[x * KW + 1] |= w[1];
  }
}

// histogram of floor(log2(count)) over rows with a nonzero sampled count
__global__ void __launch_bounds__(256) hot_hist_kernel(const uint32_t* __restrict__ cnt, uint64_t n,
                                                       unsigned long long* hist) {
  __shared__ unsigned long long h[33];
  if (threadIdx.x < 33) h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    const uint32_t c = cnt[r];
    if (c) atomicAdd(&h[31 - __clz(c)], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

// append every row whose sampled count is >= thr as (count, row)
__global__ void __launch_bounds__(256) hot_collect_kernel(const uint32_t* __restrict__ cnt, uint64_t n,
                                                          uint32_t thr, uint32_t cap, uint32_t* out,
                                                          uint32_t* out_n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    const uint32_t c = cnt[r];
    if (c >= thr) {
      const uint32_t k = atomicAdd(out_n, 1u);
      if (k < cap) {
        out[2 * k] = c;
        out[2 * k + 1] = static_cast<uint32_t>(r);
      }
    }
  }
}

__global__ void hot_map_kernel(const uint32_t* __restrict__ rows, int n, uint32_t* map) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicOr(map + (rows[i] >> 5), 1u << (rows[i] & 31));
}

unsigned grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return static_cast<unsigned>(g);
}

}  // namespace

cudaError_t launch_encode(const Layout& lay, const IdxPtrs& idx, int idx_bytes, int64_t M,
                          uint64_t* keys, int* status, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  EncodeParams ep{};
  ep.nmodes = lay.N;
  for (int n = 0; n < lay.N; ++n) {
    ep.dims[n] = lay.dims[n];
    ep.nbits[n] = lay.nbits[n];
  }
  DecodeParams dp;
  int ident[kMaxModes];
  for (int n = 0; n < kMaxModes; ++n) ident[n] = n;
  make_decode(lay, ident, &dp);
  const unsigned g = grid_for(M, 256);
  if (idx_bytes == 4) {
    if (lay.KW == 1)
      encode_kernel<uint32_t, 1><<<g, 256, 0, s>>>(dp, ep, idx, M, keys, status);
    else
      encode_kernel<uint32_t, 2><<<g, 256, 0, s>>>(dp, ep, idx, M, keys, status);
  } else {
    if (lay.KW == 1)
      encode_kernel<int64_t, 1><<<g, 256, 0, s>>>(dp, ep, idx, M, keys, status);
    else
      encode_kernel<int64_t, 2><<<g, 256, 0, s>>>(dp, ep, idx, M, keys, status);
  }
  note_launch();
  return cudaGetLastError();
}

// Stored keys: the low CW 32-bit words of every KW-word key (the index and
// its flags fit in them by construction of the layout).
__global__ void __launch_bounds__(256) pack_keys_kernel(const uint64_t* __restrict__ keys, int KW,
                                                        uint32_t* __restrict__ out, int CW, int64_t M) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < M; x += stride)
    for (int w = 0; w < CW; ++w) {
      const uint64_t k = keys[x * KW + (w >> 1)];
      out[x * CW + w] = static_cast<uint32_t>(k >> ((w & 1) * 32));
    }
}

cudaError_t launch_pack_keys(const uint64_t* keys, int KW, uint32_t* out, int CW, int64_t M, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  pack_keys_kernel<<<grid_for(M, 256), 256, 0, s>>>(keys, KW, out, CW, M);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_permute(const void* src, void* dst, const uint32_t* perm, int64_t M,
                           int elem_bytes, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const unsigned g = grid_for(M, 256);
  if (elem_bytes == 8)
    permute_kernel<uint64_t><<<g, 256, 0, s>>>(static_cast<const uint64_t*>(src),
                                               static_cast<uint64_t*>(dst), perm, M);
  else if (elem_bytes == 4)
    permute_kernel<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(src),
                                               static_cast<uint32_t*>(dst), perm, M);
  else
    permute_kernel<uint16_t><<<g, 256, 0, s>>>(static_cast<const uint16_t*>(src),
                                               static_cast<uint16_t*>(dst), perm, M);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const uint64_t* keys, int KW, const void* vals, alto_dtype vd, int64_t M,
                         double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess || M <= 0) return e;
  const unsigned g = grid_for(M, 256 * 8);
  if (vd == ALTO_F64) {
    if (KW == 1)
      sumsq_kernel<double, 1><<<g, 256, 0, s>>>(keys, static_cast<const double*>(vals), M, out);
    else
      sumsq_kernel<double, 2><<<g, 256, 0, s>>>(keys, static_cast<const double*>(vals), M, out);
  } else if (vd == ALTO_F32) {
    if (KW == 1)
      sumsq_kernel<float, 1><<<g, 256, 0, s>>>(keys, static_cast<const float*>(vals), M, out);
    else
      sumsq_kernel<float, 2><<<g, 256, 0, s>>>(keys, static_cast<const float*>(vals), M, out);
  } else {
    if (KW == 1)
      sumsq_kernel<uint16_t, 1><<<g, 256, 0, s>>>(keys, static_cast<const uint16_t*>(vals), M, out);
    else
      sumsq_kernel<uint16_t, 2><<<g, 256, 0, s>>>(keys, static_cast<const uint16_t*>(vals), M, out);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_hot_hist(const uint32_t* cnt, uint64_t n, unsigned long long* hist, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  hot_hist_kernel<<<grid_for(static_cast<int64_t>(n), 256 * 8), 256, 0, s>>>(cnt, n, hist);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_hot_collect(const uint32_t* cnt, uint64_t n, uint32_t thr, uint32_t cap, uint32_t* out,
                               uint32_t* out_n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  hot_collect_kernel<<<grid_for(static_cast<int64_t>(n), 256 * 8), 256, 0, s>>>(cnt, n, thr, cap, out, out_n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_segment_stats(const Layout& lay, const uint64_t* keys, int64_t M, int64_t L,
                                 uint32_t* ivl, uint32_t* const* first, uint32_t* const* last,
                                 uint32_t* const* cnt, cudaStream_t s) {
  if (L <= 0) return cudaSuccess;
  DecodeParams dp;
  int ident[kMaxModes];
  for (int n = 0; n < kMaxModes; ++n) ident[n] = n;
  make_decode(lay, ident, &dp);
  RowArrays ra{};
  for (int n = 0; n < lay.N; ++n) {
    ra.first[n] = first[n];
    ra.last[n] = last[n];
    ra.cnt[n] = cnt != nullptr ? cnt[n] : nullptr;
  }
  const unsigned g = grid_for(L, 8);
  if (lay.KW == 1)
    segment_stats_kernel<1><<<g, 256, 0, s>>>(dp, keys, M, L, ivl, ra);
  else
    segment_stats_kernel<2><<<g, 256, 0, s>>>(dp, keys, M, L, ivl, ra);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_count_touched(const uint32_t* first, uint64_t n, unsigned long long* out,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  count_touched_kernel<<<grid_for(static_cast<int64_t>(n), 256 * 8), 256, 0, s>>>(first, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_max_interval(const uint32_t* ivl, int64_t L, int N, unsigned long long* out,
                                cudaStream_t s) {
  if (L <= 0) return cudaSuccess;
  max_interval_kernel<<<grid_for(L * N, 256), 256, 0, s>>>(ivl, L, N, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_hot_map(const uint32_t* rows, int n, uint32_t* map, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  hot_map_kernel<<<(n + 255) / 256, 256, 0, s>>>(rows, n, map);
  note_launch();
  return cudaGetLastError();
}

// One pass per kind of flag: the boundary / internal flags of Sec. 3.3
// (hotmap == nullptr) or the hot-row flags (hotmap given per mode).
cudaError_t launch_set_flags(const Layout& lay, uint64_t* keys, int64_t M,
                             uint32_t* const* first, uint32_t* const* last,
                             uint32_t* const* hotmap, cudaStream_t s) {
  FlagParams fp{};
  fp.hot = hotmap != nullptr ? 1 : 0;
  for (int n = 0; n < lay.N; ++n) {
    const int b = fp.hot ? lay.hot_bit[n] : lay.flag_bit[n];
    if (b >= 0 && (!fp.hot || hotmap[n] != nullptr)) {
      fp.slot[fp.nflag] = n;
      fp.bit[fp.nflag] = b;
      if (fp.hot) fp.map[fp.nflag] = hotmap[n];
      fp.nflag++;
    }
  }
  if (fp.nflag == 0 || M <= 0) return cudaSuccess;
  DecodeParams dp;
  int ident[kMaxModes];
  for (int n = 0; n < kMaxModes; ++n) ident[n] = n;
  make_decode(lay, ident, &dp);
  RowArrays ra{};
  for (int n = 0; n < lay.N; ++n) {
    ra.first[n] = first[n];
    ra.last[n] = last[n];
  }
  const unsigned g = grid_for(M, 256);
  if (lay.KW == 1)
    set_flags_kernel<1><<<g, 256, 0, s>>>(dp, fp, keys, M, ra);
  else
    set_flags_kernel<2><<<g, 256, 0, s>>>(dp, fp, keys, M, ra);
  note_launch();
  return cudaGetLastError();
}

}  // namespace alto
