// Device-side building blocks shared by the libalto kernels: key access,
// bit-level de-linearization (Sec. 3.1, EXTRACT of Alg. 1-2), the device
// status word, and vector atomics.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "alto.h"

namespace alto {

constexpr int kMaxModes = ALTO_MAX_MODES;

// ---------------------------------------------------------------------------
// De-linearization parameters.
//
// A key of KW 64-bit words is viewed as 2*KW 32-bit words.  For every mode
// slot s and 32-bit word w, mask[s][w] holds the key bits of that word that
// belong to the mode, and the mode's bits in that word are compacted with
// the five-step parallel-suffix "compress" (Hacker's Delight, 2nd ed.,
// Sec. 7-4): x &= mask; for i in 0..4: t = x & mv[i]; x = (x ^ t) | (t >> 2^i).
// The move masks mv depend only on the mask and are precomputed on the host.
// The compacted word is shifted left by shift[s][w], the number of the
// mode's bits held in lower words (a mode's bits ascend with key position,
// so lower words hold its low-order bits).
//
// Slots are an ordering of the modes chosen by the caller (MTTKRP puts the
// output mode in the last slot); mode_of[s] records which mode a slot is.
struct DecodeParams {
  int nmodes;
  int words32;
  int mode_of[kMaxModes];
  uint32_t mask[kMaxModes][4];
  uint32_t mv[kMaxModes][4][5];
  uint32_t shift[kMaxModes][4];
};

template <int KW>
struct KeyT {
  uint32_t w[2 * KW];
};

template <int KW>
__device__ __forceinline__ KeyT<KW> load_key(const uint64_t* keys, int64_t x) {
  KeyT<KW> k;
  if constexpr (KW == 1) {
    uint2 v = __ldcs(reinterpret_cast<const uint2*>(keys) + x);
    k.w[0] = v.x;
    k.w[1] = v.y;
  } else {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(keys) + x);
    k.w[0] = v.x;
    k.w[1] = v.y;
    k.w[2] = v.z;
    k.w[3] = v.w;
  }
  return k;
}

// Index of the mode in slot s.  Words without bits of the mode are skipped
// (the test is uniform across the warp).
template <int KW>
__device__ __forceinline__ uint32_t extract(const KeyT<KW>& k, const DecodeParams& p, int s) {
  uint32_t r = 0;
#pragma unroll
  for (int w = 0; w < 2 * KW; ++w) {
    const uint32_t m = p.mask[s][w];
    if (m != 0u) {
      uint32_t x = k.w[w] & m;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const uint32_t t = x & p.mv[s][w][i];
        x = (x ^ t) | (t >> (1u << i));
      }
      r |= x << p.shift[s][w];
    }
  }
  return r;
}

// ---------------------------------------------------------------------------
// The stored (MTTKRP) form of a key: the ALTO index and its flag bits in the
// fewest 32-bit words, W in 1..4 (Sec. 4.2.3 uses multiples of the native
// word; 32 and 96 bits are the packed widths), word 0 holding the lowest
// bits.  Key x occupies words [W x, W x + W).
template <int W>
struct CKey {
  uint32_t w[W];
};

template <int W>
__device__ __forceinline__ CKey<W> load_ckey(const uint32_t* keys, int64_t x) {
  CKey<W> k;
  if constexpr (W == 1) {
    k.w[0] = __ldcs(keys + x);
  } else if constexpr (W == 2) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(keys) + x);
    k.w[0] = v.x;
    k.w[1] = v.y;
  } else if constexpr (W == 3) {  // 12-byte keys: three 4-byte loads (the warp's 384 bytes are contiguous)
    const uint32_t* p = keys + 3 * x;
    k.w[0] = __ldcs(p);
    k.w[1] = __ldcs(p + 1);
    k.w[2] = __ldcs(p + 2);
  } else {
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(keys) + x);
    k.w[0] = v.x;
    k.w[1] = v.y;
    k.w[2] = v.z;
    k.w[3] = v.w;
  }
  return k;
}

// Index of the mode in slot s from a stored key (EXTRACT of Alg. 1-2): the
// five-step compress of every word holding bits of the mode.
template <int W>
__device__ __forceinline__ uint32_t extract_c(const CKey<W>& k, const DecodeParams& p, int s) {
  uint32_t r = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t m = p.mask[s][w];
    if (m != 0u) {
      uint32_t x = k.w[w] & m;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const uint32_t t = x & p.mv[s][w][i];
        x = (x ^ t) | (t >> (1u << i));
      }
      r |= x << p.shift[s][w];
    }
  }
  return r;
}

template <int W>
__device__ __forceinline__ uint32_t ckey_bit(const CKey<W>& k, int bit) {
  uint32_t w = k.w[0];
#pragma unroll
  for (int i = 1; i < W; ++i)
    if ((bit >> 5) == i) w = k.w[i];
  return (w >> (bit & 31)) & 1u;
}

// First position of line segment l of L over M nonzeros: floor(l * M / L)
// (Sec. 3.2), in unsigned 64-bit arithmetic (M < 2^32, l <= L <= M).
__host__ __device__ __forceinline__ int64_t seg_begin(int64_t l, int64_t M, int64_t L) {
  return static_cast<int64_t>(static_cast<uint64_t>(l) * static_cast<uint64_t>(M) /
                              static_cast<uint64_t>(L));
}

// Bit `bit` of a key (selects between the 32-bit words without indexing
// the register array dynamically).
template <int KW>
__device__ __forceinline__ uint32_t key_bit(const KeyT<KW>& k, int bit) {
  uint32_t w = k.w[0];
#pragma unroll
  for (int i = 1; i < 2 * KW; ++i)
    if ((bit >> 5) == i) w = k.w[i];
  return (w >> (bit & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Device status word: the first error recorded wins.
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status != nullptr) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Fire-and-forget vector atomics into global memory (RED; no return value).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

__device__ __forceinline__ void red_add_f64(double* addr, double a) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(a) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace alto
