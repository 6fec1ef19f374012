// Ordering stage of ALTO generation (Sec. 3.1): stable ascending sort of the
// linearized keys, carrying each nonzero's input position.
//
// LSD radix sort, 8-bit digits, only over the bits the index uses.  Every
// pass runs three kernels:
//   1. tile histogram  -- per 4096-key tile, count of each digit, stored
//                         digit-major: counts[digit * ntiles + tile];
//   2. exclusive scan  -- over that array, giving every (digit, tile) its
//                         first output slot;
//   3. scatter         -- each tile ranks its keys stably (warp match on the
//                         digit inside 32-key rounds, running per-warp digit
//                         counts, then a prefix over the tile's warps),
//                         stages them in shared memory in digit order and
//                         writes every digit's run out contiguously.
// Equal keys keep their input order (LSD passes are each stable), which is
// what the ordering stage needs when duplicates are present.  The passes
// never wait on one another inside a kernel, so no device spin is needed.
#include "internal.h"

namespace alto {

namespace {

constexpr int kDigitBits = kSortDigitBits;
constexpr int kRadix = 1 << kDigitBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 16;                       // keys per lane
constexpr int kTile = kSortThreads * kItems;     // 4096 keys per tile
constexpr int kWarpItems = kTile / kSortWarps;   // 512 keys per warp

template <int KW>
__device__ __forceinline__ uint32_t digit_of(const uint64_t* k, int shift) {
  if constexpr (KW == 1) {
    return static_cast<uint32_t>(k[0] >> shift) & (kRadix - 1);
  } else {
    return shift < 64 ? static_cast<uint32_t>(k[0] >> shift) & (kRadix - 1)
                      : static_cast<uint32_t>(k[1] >> (shift - 64)) & (kRadix - 1);
  }
}

template <int KW>
__global__ void __launch_bounds__(kSortThreads) tile_histogram(const uint64_t* __restrict__ keys,
                                                               int64_t M, int shift, int64_t ntiles,
                                                               uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[kSortWarps][kRadix];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int64_t base = tile * kTile;
  for (int j = threadIdx.x; j < kTile; j += kSortThreads) {
    const int64_t x = base + j;
    if (x < M) {
      uint64_t k[KW];
#pragma unroll
      for (int w = 0; w < KW; ++w) k[w] = __ldcs(keys + x * KW + w);
      atomicAdd(&h[warp][digit_of<KW>(k, shift)], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
    counts[static_cast<int64_t>(d) * ntiles + tile] = s;
  }
}

template <int KW>
__global__ void __launch_bounds__(kSortThreads) tile_scatter(
    const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ perm_in,
    uint64_t* __restrict__ keys_out, uint32_t* __restrict__ perm_out, int64_t M, int shift,
    int64_t ntiles, const uint32_t* __restrict__ offsets, int iota_perm) {
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t tstart[kRadix];   // first staged slot of each digit
  __shared__ uint32_t gbase[kRadix];    // first output slot of each digit for this tile
  extern __shared__ __align__(16) unsigned char stage_raw[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(stage_raw);             // kTile x KW
  uint32_t* sperm = reinterpret_cast<uint32_t*>(skey + kTile * KW);   // kTile
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int64_t wbase = tile * kTile + static_cast<int64_t>(warp) * kWarpItems;

  uint64_t k[kItems][KW];
  uint32_t pv[kItems];
  uint32_t dg[kItems];
  uint32_t local[kItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t x = wbase + r * 32 + lane;
    const bool ok = x < M;
    if (ok) {
#pragma unroll
      for (int w = 0; w < KW; ++w) k[r][w] = __ldcs(keys_in + x * KW + w);
      pv[r] = iota_perm ? static_cast<uint32_t>(x) : __ldcs(perm_in + x);
      dg[r] = digit_of<KW>(k[r], shift);
    } else {
#pragma unroll
      for (int w = 0; w < KW; ++w) k[r][w] = 0;
      pv[r] = 0;
      dg[r] = kRadix + lane;  // unique, never matches a real digit
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, dg[r]);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (ok) base = wcnt[warp][dg[r]];
    __syncwarp();
    if (ok && lane == leader) wcnt[warp][dg[r]] = base + __popc(peers);
    __syncwarp();
    local[r] = base + __popc(peers & lt);
  }
  __syncthreads();
  // exclusive prefix over the tile's warps, per digit (in place); digit totals
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = s;
      s += c;
    }
    tstart[d] = s;  // total of digit d (turned into a start below)
    gbase[d] = offsets[static_cast<int64_t>(d) * ntiles + tile];
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the 256 digit totals by one warp
    uint32_t v[kRadix / 32];
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < kRadix / 32; ++q) {
      v[q] = tstart[threadIdx.x * (kRadix / 32) + q];
      run += v[q];
    }
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (threadIdx.x >= o) inc += y;
    }
    uint32_t base = inc - run;
#pragma unroll
    for (int q = 0; q < kRadix / 32; ++q) {
      tstart[threadIdx.x * (kRadix / 32) + q] = base;
      base += v[q];
    }
  }
  __syncthreads();
  // stage in digit order
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t x = wbase + r * 32 + lane;
    if (x < M) {
      const uint32_t d = dg[r];
      const uint32_t pos = tstart[d] + wcnt[warp][d] + local[r];
#pragma unroll
      for (int w = 0; w < KW; ++w) skey[pos * KW + w] = k[r][w];
      sperm[pos] = pv[r];
    }
  }
  __syncthreads();
  // write out: consecutive staged slots of one digit go to consecutive slots
  const int64_t tbase = tile * kTile;
  const int n = static_cast<int>(M - tbase < kTile ? M - tbase : kTile);
  for (int i = threadIdx.x; i < n; i += kSortThreads) {
    uint64_t kk[KW];
#pragma unroll
    for (int w = 0; w < KW; ++w) kk[w] = skey[i * KW + w];
    const uint32_t d = digit_of<KW>(kk, shift);
    const int64_t dst = static_cast<int64_t>(gbase[d]) + (i - tstart[d]);
#pragma unroll
    for (int w = 0; w < KW; ++w) keys_out[dst * KW + w] = kk[w];
    perm_out[dst] = sperm[i];
  }
}

// --- exclusive scan of uint32 (reduce, scan block sums, apply) -----------
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < kScanThreads / 32) ? wsum[lane] : 0;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kScanThreads / 32) wsum[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint32_t r = wsum[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                           uint32_t* __restrict__ part) {
  __shared__ uint32_t total;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk + threadIdx.x * kScanPer;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j)
    if (base + j < n) s += in[base + j];
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_parts(uint32_t* __restrict__ part, int64_t nparts) {
  __shared__ uint32_t total;
  uint32_t carry = 0;
  for (int64_t b = 0; b < nparts; b += kScanThreads) {
    const int64_t i = b + threadIdx.x;
    const uint32_t v = i < nparts ? part[i] : 0;
    const uint32_t ex = block_exclusive_scan(v, &total);
    if (i < nparts) part[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply(const uint32_t* __restrict__ in, int64_t n,
                                                          const uint32_t* __restrict__ part,
                                                          uint32_t* __restrict__ out) {
  __shared__ uint32_t total;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk + threadIdx.x * kScanPer;
  uint32_t v[kScanPer];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    v[j] = (base + j < n) ? in[base + j] : 0;
    s += v[j];
  }
  uint32_t run = block_exclusive_scan(s, &total) + part[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
}

}  // namespace

static_assert(kTile == 4096 && kRadix == 256 && kScanChunk == 8192, "sort_scratch_words_for layout");

int64_t sort_scratch_words(int64_t M) { return sort_scratch_words_for(M); }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  scan_reduce<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, part);
  scan_parts<<<1, kScanThreads, 0, s>>>(part, nb);
  scan_apply<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, part, out);
  note_launch(3);
  return cudaGetLastError();
}

cudaError_t radix_sort_pairs(uint64_t** keys, uint64_t** keys_alt, uint32_t** perm,
                             uint32_t** perm_alt, int64_t M, int KW, int nbits, uint32_t* scratch,
                             cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const int64_t ntiles = (M + kTile - 1) / kTile;
  const int64_t ncount = ntiles * kRadix;
  uint32_t* counts = scratch;
  uint32_t* offsets = scratch + ncount;
  uint32_t* part = scratch + 2 * ncount;
  const int passes = sort_passes_for(nbits);
  bool iota = true;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kDigitBits;
    if (KW == 1) {
      tile_histogram<1><<<static_cast<unsigned>(ntiles), kSortThreads, 0, s>>>(*keys, M, shift, ntiles,
                                                                               counts);
    } else {
      tile_histogram<2><<<static_cast<unsigned>(ntiles), kSortThreads, 0, s>>>(*keys, M, shift, ntiles,
                                                                               counts);
    }
    cudaError_t e = exclusive_scan_u32(counts, offsets, ncount, part, s);
    if (e != cudaSuccess) return e;
    const size_t stage = static_cast<size_t>(kTile) * (8 * KW + 4);
    if (KW == 1) {
      if (p == 0) cudaFuncSetAttribute(tile_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(stage));
      tile_scatter<1><<<static_cast<unsigned>(ntiles), kSortThreads, stage, s>>>(
          *keys, *perm, *keys_alt, *perm_alt, M, shift, ntiles, offsets, iota ? 1 : 0);
    } else {
      if (p == 0) cudaFuncSetAttribute(tile_scatter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(stage));
      tile_scatter<2><<<static_cast<unsigned>(ntiles), kSortThreads, stage, s>>>(
          *keys, *perm, *keys_alt, *perm_alt, M, shift, ntiles, offsets, iota ? 1 : 0);
    }
    note_launch(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    iota = false;
    uint64_t* tk = *keys;
    *keys = *keys_alt;
    *keys_alt = tk;
    uint32_t* tp = *perm;
    *perm = *perm_alt;
    *perm_alt = tp;
  }
  return cudaSuccess;
}

}  // namespace alto
