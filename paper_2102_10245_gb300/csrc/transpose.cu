// Sparse tensor transposition over the ALTO format (Sec. 5, sparse tensor
// operations): the nonzeros are put in the lexicographic order of a chosen
// sequence of modes.  Transposition reduces to sorting by the coordinates of
// the new mode order; the linearized index already holds every coordinate
// bit, so the sort key is cut straight out of the stored key and the LSD
// radix sort runs over the chosen modes' bits only -- a partial radix sort
// (sum of b_m over the chosen modes, not all B index bits).  The sort starts
// from ALTO order and every pass is stable, so nonzeros that tie on the
// chosen modes stay in ALTO order (and duplicates in input order).
//
//   1. transpose_key_kernel    stored key -> concatenated key of the chosen
//                              modes' coordinates (first chosen mode in the
//                              most significant bits)
//   2. radix_sort_pairs        stable LSD sort of (key, ALTO position) over
//                              those bits
//   3. transpose_gather_kernel result: ALTO position, input position,
//                              coordinates in the new mode order, value
#include "internal.h"

namespace alto {

namespace {

constexpr int kTThreads = 256;

struct TKeyParams {
  int nsel;          // chosen modes (decode slots 0..nsel-1)
  int kw;            // 64-bit words of the sort key (1 or 2)
  int off[kMaxModes];  // bit offset of slot j in the sort key
};

template <int CW>
__global__ void __launch_bounds__(kTThreads) transpose_key_kernel(const __grid_constant__ DecodeParams dp,
                                                                  const __grid_constant__ TKeyParams kp,
                                                                  const uint32_t* __restrict__ ckeys, int64_t M,
                                                                  uint64_t* __restrict__ out) {
  for (int64_t x = blockIdx.x * static_cast<int64_t>(kTThreads) + threadIdx.x; x < M;
       x += static_cast<int64_t>(gridDim.x) * kTThreads) {
    const CKey<CW> k = load_ckey<CW>(ckeys, x);
    uint64_t w0 = 0, w1 = 0;
    for (int j = 0; j < kp.nsel; ++j) {
      const uint64_t id = extract_c<CW>(k, dp, j);
      const int o = kp.off[j];
      if (o >= 64) {
        w1 |= id << (o - 64);
      } else {
        w0 |= id << o;
        if (o > 32) w1 |= id >> (64 - o);  // coordinates have at most 32 bits
      }
    }
    if (kp.kw == 1) {
      out[x] = w0;
    } else {
      out[2 * x] = w0;
      out[2 * x + 1] = w1;
    }
  }
}

struct TGatherParams {
  int N;
  int nsel;
  int kw;
  int idx_bytes;     // 4 or 8
  int vbytes;        // 2, 4 or 8
  int off[kMaxModes];
  uint32_t omask[kMaxModes];  // (1 << b) - 1 of output mode j (all ones for 32 bits)
  void* idx[kMaxModes];       // output coordinate arrays (output mode order), or null
};

template <int CW>
__global__ void __launch_bounds__(kTThreads) transpose_gather_kernel(
    const __grid_constant__ DecodeParams dp, const __grid_constant__ TGatherParams gp,
    const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ ckeys,
    const uint32_t* __restrict__ perm, const void* __restrict__ vals, int64_t M, uint32_t* __restrict__ order,
    uint32_t* __restrict__ src, void* __restrict__ vout) {
  for (int64_t y = blockIdx.x * static_cast<int64_t>(kTThreads) + threadIdx.x; y < M;
       y += static_cast<int64_t>(gridDim.x) * kTThreads) {
    const uint32_t q = sorted[y];
    if (order != nullptr) order[y] = q;
    if (src != nullptr) src[y] = __ldg(perm + q);
    if (vout != nullptr) {
      if (gp.vbytes == 8)
        static_cast<uint64_t*>(vout)[y] = __ldg(static_cast<const unsigned long long*>(vals) + q);
      else if (gp.vbytes == 4)
        static_cast<uint32_t*>(vout)[y] = __ldg(static_cast<const unsigned int*>(vals) + q);
      else
        static_cast<uint16_t*>(vout)[y] = __ldg(static_cast<const unsigned short*>(vals) + q);
    }
    if (gp.idx[0] == nullptr) continue;
    // chosen modes: cut out of the sorted key (read in order); the rest:
    // de-linearized from the stored key of ALTO position q
    const uint64_t w0 = gp.kw == 2 ? skeys[2 * y] : skeys[y];
    const uint64_t w1 = gp.kw == 2 ? skeys[2 * y + 1] : 0ull;
    CKey<CW> k{};
    if (gp.nsel < gp.N) k = load_ckey<CW>(ckeys, q);
    for (int j = 0; j < gp.N; ++j) {
      uint32_t id;
      if (j < gp.nsel) {
        const int o = gp.off[j];
        const uint64_t v = o >= 64 ? (w1 >> (o - 64)) : (o == 0 ? w0 : ((w0 >> o) | (w1 << (64 - o))));
        id = static_cast<uint32_t>(v) & gp.omask[j];
      } else {
        id = extract_c<CW>(k, dp, j);
      }
      if (gp.idx_bytes == 8)
        static_cast<int64_t*>(gp.idx[j])[y] = static_cast<int64_t>(id);
      else
        static_cast<uint32_t*>(gp.idx[j])[y] = id;
    }
  }
}

unsigned grid_for(int64_t M) {
  const int64_t b = (M + kTThreads - 1) / kTThreads;
  return static_cast<unsigned>(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

template <int CW>
void launch_keys(const DecodeParams& dp, const TKeyParams& kp, const uint32_t* ckeys, int64_t M, uint64_t* out,
                 cudaStream_t s) {
  transpose_key_kernel<CW><<<grid_for(M), kTThreads, 0, s>>>(dp, kp, ckeys, M, out);
}

template <int CW>
void launch_gather(const DecodeParams& dp, const TGatherParams& gp, const uint64_t* skeys, const uint32_t* sorted,
                   const uint32_t* ckeys, const uint32_t* perm, const void* vals, int64_t M, uint32_t* order,
                   uint32_t* src, void* vout, cudaStream_t s) {
  transpose_gather_kernel<CW><<<grid_for(M), kTThreads, 0, s>>>(dp, gp, skeys, sorted, ckeys, perm, vals, M,
                                                                order, src, vout);
}

}  // namespace

}  // namespace alto

using namespace alto;

alto_status alto_transpose(alto_t t, int nsel, const int* modes, uint32_t* order, uint32_t* src, void* const* idx,
                           int idx_bytes, void* vals, void* stream) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  const Layout& lay = t->lay;
  const int N = lay.N;
  if (nsel < 1 || nsel > N || modes == nullptr) return fail(ALTO_EINVAL, "nsel %d outside [1, %d]", nsel, N);
  if (idx != nullptr && idx_bytes != 4 && idx_bytes != 8) return fail(ALTO_EINVAL, "idx_bytes must be 4 or 8");
  bool used[kMaxModes] = {};
  int slot_mode[kMaxModes];
  for (int j = 0; j < nsel; ++j) {
    if (modes[j] < 0 || modes[j] >= N || used[modes[j]]) return fail(ALTO_EINVAL, "bad or repeated mode %d", modes[j]);
    used[modes[j]] = true;
    slot_mode[j] = modes[j];
  }
  int k = nsel;
  for (int m = 0; m < N; ++m)
    if (!used[m]) slot_mode[k++] = m;
  const int64_t M = t->M;
  if (M == 0) return ALTO_OK;
  if (idx != nullptr)
    for (int j = 0; j < N; ++j)
      if (idx[j] == nullptr) return fail(ALTO_EINVAL, "null coordinate output %d", j);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  DecodeParams dp;
  make_decode(lay, slot_mode, &dp);
  TKeyParams kp{};
  TGatherParams gp{};
  int bits = 0;
  for (int j = nsel - 1; j >= 0; --j) {
    kp.off[j] = gp.off[j] = bits;
    bits += lay.nbits[slot_mode[j]];
  }
  kp.nsel = gp.nsel = nsel;
  kp.kw = gp.kw = bits > 64 ? 2 : 1;
  gp.N = N;
  gp.idx_bytes = idx_bytes;
  gp.vbytes = t->vdtype == ALTO_F64 ? 8 : (t->vdtype == ALTO_F32 ? 4 : 2);
  for (int j = 0; j < N; ++j) {
    const int b = lay.nbits[slot_mode[j]];
    gp.omask[j] = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
    gp.idx[j] = idx != nullptr ? idx[j] : nullptr;
  }
  const int KWn = kp.kw;

  alto_status st = ALTO_OK;
  uint64_t* keys = nullptr;
  uint64_t* keys_alt = nullptr;
  uint32_t* perm = nullptr;
  uint32_t* perm_alt = nullptr;
  uint32_t* scratch = nullptr;
  cudaError_t e = cudaSuccess;
  keys = static_cast<uint64_t*>(dev_alloc(t, sizeof(uint64_t) * KWn * M));
  keys_alt = static_cast<uint64_t*>(dev_alloc(t, sizeof(uint64_t) * KWn * M));
  perm = static_cast<uint32_t*>(dev_alloc(t, sizeof(uint32_t) * M));
  perm_alt = static_cast<uint32_t*>(dev_alloc(t, sizeof(uint32_t) * M));
  scratch = static_cast<uint32_t*>(dev_alloc(t, sizeof(uint32_t) * sort_scratch_words(M)));
  if (!keys || !keys_alt || !perm || !perm_alt || !scratch) {
    st = fail(ALTO_ENOMEM, "transpose scratch allocation failed");
  } else {
    switch (lay.CW) {
      case 1: launch_keys<1>(dp, kp, t->ckeys, M, keys, s); break;
      case 2: launch_keys<2>(dp, kp, t->ckeys, M, keys, s); break;
      case 3: launch_keys<3>(dp, kp, t->ckeys, M, keys, s); break;
      default: launch_keys<4>(dp, kp, t->ckeys, M, keys, s); break;
    }
    note_launch();
    e = cudaGetLastError();
    // the sort writes the ALTO positions itself in its first pass
    if (e == cudaSuccess) e = radix_sort_pairs(&keys, &keys_alt, &perm, &perm_alt, M, KWn, bits, scratch, s);
    if (e == cudaSuccess) {
      switch (lay.CW) {
        case 1: launch_gather<1>(dp, gp, keys, perm, t->ckeys, t->perm, t->vals, M, order, src, vals, s); break;
        case 2: launch_gather<2>(dp, gp, keys, perm, t->ckeys, t->perm, t->vals, M, order, src, vals, s); break;
        case 3: launch_gather<3>(dp, gp, keys, perm, t->ckeys, t->perm, t->vals, M, order, src, vals, s); break;
        default: launch_gather<4>(dp, gp, keys, perm, t->ckeys, t->perm, t->vals, M, order, src, vals, s); break;
      }
      note_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = fail(ALTO_ECUDA, "transpose: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(s);  // the temporaries are freed below
  dev_free(t, keys);
  dev_free(t, keys_alt);
  dev_free(t, perm);
  dev_free(t, perm_alt);
  dev_free(t, scratch);
  return st;
}
