// Host side of the ALTO index layout (Sec. 3.1, Eq. 1): bits per mode, the
// level-by-level bit assignment, key width, and the precomputed masks that
// the device uses for de-linearization.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace alto {

namespace {

int bits_for_length(uint64_t I) {
  int b = 0;
  while (b < 64 && (1ull << b) < I) ++b;
  return b;
}

// Move masks of the five-step parallel-suffix compress of `m`
// (Hacker's Delight, 2nd ed., Sec. 7-4).
void compress_moves(uint32_t m, uint32_t mv[5]) {
  uint32_t mk = ~m << 1;
  for (int i = 0; i < 5; ++i) {
    uint32_t mp = mk ^ (mk << 1);
    mp ^= mp << 2;
    mp ^= mp << 4;
    mp ^= mp << 8;
    mp ^= mp << 16;
    const uint32_t v = mp & m;
    mv[i] = v;
    m = (m ^ v) | (v >> (1u << i));
    mk = mk & ~mp;
  }
}

uint32_t apply_compress(uint32_t x, uint32_t m, const uint32_t mv[5]) {
  x &= m;
  for (int i = 0; i < 5; ++i) {
    const uint32_t t = x & mv[i];
    x = (x ^ t) | (t >> (1u << i));
  }
  return x;
}

}  // namespace

// Bits per mode b_n = ceil(log2 I_n); walking levels l = 0, 1, ... from the
// least significant key bit, and inside a level the modes in increasing
// order of length (ties: lower mode first), each mode with l < b_n takes
// the next key bit.  Key width: the smallest of 64 / 128 bits that holds the
// index (Sec. 4.2.3), unless key_bits forces one.
alto_status make_layout(int N, const uint64_t* dims, int key_bits, Layout* out) {
  Layout L;
  if (N < 1 || N > kMaxModes) return fail(ALTO_EINVAL, "nmodes %d outside [1, %d]", N, kMaxModes);
  L.N = N;
  int maxb = 0;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1 || dims[n] > (1ull << 32))
      return fail(ALTO_EINVAL, "mode %d length %llu outside [1, 2^32]", n,
                  static_cast<unsigned long long>(dims[n]));
    L.dims[n] = dims[n];
    L.nbits[n] = bits_for_length(dims[n]);
    maxb = std::max(maxb, L.nbits[n]);
    L.flag_bit[n] = -1;
    L.hot_bit[n] = -1;
  }
  int order[kMaxModes];
  for (int n = 0; n < N; ++n) order[n] = n;
  std::stable_sort(order, order + N, [&](int a, int b) { return dims[a] < dims[b]; });
  int next = 0;
  for (int l = 0; l < maxb; ++l)
    for (int a = 0; a < N; ++a) {
      const int n = order[a];
      if (l < L.nbits[n]) {
        L.pos[n][l] = next;
        L.mask[n][next >> 6] |= 1ull << (next & 63);
        ++next;
      }
    }
  L.B = next;
  if (next > 128) return fail(ALTO_EOVERFLOW, "index needs %d bits (> 128)", next);
  if (key_bits == 0) {
    L.KW = next <= 64 ? 1 : 2;
  } else if (key_bits == 64) {
    if (next > 64) return fail(ALTO_EOVERFLOW, "index needs %d bits, 64-bit key requested", next);
    L.KW = 1;
  } else if (key_bits == 128) {
    L.KW = 2;
  } else {
    return fail(ALTO_EINVAL, "key_bits must be 0, 64 or 128 (got %d)", key_bits);
  }
  // stored key width: the fewest 32-bit words that hold the index (1..4),
  // unless key_bits forces the full 64- or 128-bit word
  if (key_bits == 0) {
    L.CW = next > 0 ? (next + 31) / 32 : 1;
    if (L.CW > 2 * L.KW) L.CW = 2 * L.KW;
  } else {
    L.CW = 2 * L.KW;
  }
  *out = L;
  return ALTO_OK;
}

void make_decode(const Layout& lay, const int* slot_mode, DecodeParams* dp) {
  std::memset(dp, 0, sizeof(*dp));
  dp->nmodes = lay.N;
  dp->words32 = lay.CW;
  for (int s = 0; s < lay.N; ++s) {
    const int n = slot_mode[s];
    dp->mode_of[s] = n;
    uint32_t below = 0;
    for (int w = 0; w < 2 * lay.KW; ++w) {
      const uint32_t m = static_cast<uint32_t>(lay.mask[n][w >> 1] >> ((w & 1) * 32));
      dp->mask[s][w] = m;
      compress_moves(m, dp->mv[s][w]);
      dp->shift[s][w] = below;
      below += static_cast<uint32_t>(__builtin_popcount(m));
    }
  }
}

// Host de-linearization with the same masks as the device.
void host_decode(const Layout& lay, const uint64_t* key, uint32_t* idx) {
  DecodeParams dp;
  int ident[kMaxModes];
  for (int n = 0; n < kMaxModes; ++n) ident[n] = n;
  make_decode(lay, ident, &dp);
  for (int s = 0; s < lay.N; ++s) {
    uint32_t r = 0;
    for (int w = 0; w < 2 * lay.KW; ++w) {
      const uint32_t kw = static_cast<uint32_t>(key[w >> 1] >> ((w & 1) * 32));
      if (dp.mask[s][w]) r |= apply_compress(kw, dp.mask[s][w], dp.mv[s][w]) << dp.shift[s][w];
    }
    idx[s] = r;
  }
}

}  // namespace alto
