// C ABI of libalto (declared in include/alto.h): argument checking, input
// staging, ALTO generation (Sec. 3.1-3.3), statistics, and the MTTKRP and
// CP-ALS entry points.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace {

thread_local char g_err[512] = "";
std::atomic<uint64_t> g_launches{0};

constexpr int64_t kSegNnz = 2048;    // default nonzeros per line segment
constexpr int64_t kMinSegNnz = 256;  // smallest automatic segment

// Automatic L: segments of kSegNnz nonzeros, halved (down to kMinSegNnz)
// while the tensor would give fewer than two thread-block units per SM, so
// that small tensors still spread over the GPU.
int64_t auto_segments(int64_t nnz) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  int64_t seg = kSegNnz;
  const int64_t unit = alto::kUnitSegs;
  while (seg > kMinSegNnz && (nnz + seg * unit - 1) / (seg * unit) < 2 * static_cast<int64_t>(sms)) seg >>= 1;
  return (nnz + seg - 1) / seg;
}

}  // namespace

namespace alto {

alto_status fail(alto_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void note_launch(int k) { g_launches.fetch_add(static_cast<uint64_t>(k), std::memory_order_relaxed); }
uint64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t prof_begin(alto_tensor_s* t, int mode, cudaStream_t s) {
  if (!t->prof) return cudaSuccess;
  while (t->ev_pool.size() < 2 * (t->ev_used + 1)) {
    cudaEvent_t e;
    const cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    t->ev_pool.push_back(e);
  }
  if (t->ev_mode.size() < t->ev_used + 1) t->ev_mode.resize(t->ev_used + 1);
  t->ev_mode[t->ev_used] = mode;
  return cudaEventRecord(t->ev_pool[2 * t->ev_used], s);
}

cudaError_t prof_end(alto_tensor_s* t, cudaStream_t s) {
  if (!t->prof) return cudaSuccess;
  const cudaError_t r = cudaEventRecord(t->ev_pool[2 * t->ev_used + 1], s);
  t->ev_used++;
  return r;
}

void* dev_alloc(alto_tensor_s* t, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~static_cast<size_t>(255);
  if (t->alloc_fn != nullptr) return t->alloc_fn(bytes, t->alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(alto_tensor_s* t, void* p) {
  if (p == nullptr) return;
  if (t->free_fn != nullptr)
    t->free_fn(p, t->alloc_ctx);
  else
    cudaFree(p);
}

}  // namespace alto

using namespace alto;

#define CK(expr)                                                                            \
  do {                                                                                      \
    const cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) {                                                                \
      st = fail(ALTO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                       \
      goto done;                                                                            \
    }                                                                                       \
  } while (0)

#define ALLOC(ptr, type, bytes)                                                             \
  do {                                                                                      \
    ptr = static_cast<type>(dev_alloc(t, (bytes)));                                         \
    if (ptr == nullptr) {                                                                   \
      st = fail(ALTO_ENOMEM, "device allocation of %zu bytes failed", static_cast<size_t>(bytes)); \
      goto done;                                                                            \
    }                                                                                       \
  } while (0)

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_format(alto_tensor_s* t) {
  if (t->ckeys != reinterpret_cast<uint32_t*>(t->keys)) dev_free(t, t->ckeys);
  t->ckeys = nullptr;
  dev_free(t, t->keys);
  dev_free(t, t->perm);
  dev_free(t, t->vals);
  dev_free(t, t->ivl);
  dev_free(t, t->status);
  for (int n = 0; n < kMaxModes; ++n) {
    dev_free(t, t->hot[n]);
    t->hot[n] = nullptr;
    t->hot_n[n] = 0;
  }
  dev_free(t, t->hot_rep);
  t->hot_rep = nullptr;
  t->hot_rep_bytes = 0;
  t->keys = nullptr;
  t->perm = nullptr;
  t->vals = nullptr;
  t->ivl = nullptr;
  t->status = nullptr;
  for (int n = 0; n < kMaxModes; ++n) free_temp_plan(t, n);
  CpalsWork& w = t->cp;
  dev_free(t, w.mt);
  dev_free(t, w.atmp);
  dev_free(t, w.gram);
  dev_free(t, w.vinv64);
  dev_free(t, w.vinv32);
  dev_free(t, w.colstat);
  dev_free(t, w.scal);
  dev_free(t, w.fits);
  w = CpalsWork();
  for (cudaEvent_t e : t->ev_pool) cudaEventDestroy(e);
  t->ev_pool.clear();
  t->ev_mode.clear();
  t->ev_used = 0;
}

// Union of the intervals of every 8 consecutive segments (one thread-block
// unit), per mode.
void unit_intervals(alto_tensor_s* t, const std::vector<uint32_t>& ivl) {
  const int N = t->lay.N;
  const int64_t L = t->L;
  const int64_t U = (L + 7) / 8;
  for (int n = 0; n < N; ++n) {
    t->unit_lo[n].assign(U, 1);
    t->unit_hi[n].assign(U, 0);
    t->unit_width_sorted[n].resize(U);
    for (int64_t u = 0; u < U; ++u) {
      uint32_t lo = 0xffffffffu, hi = 0;
      bool any = false;
      for (int64_t l = u * 8; l < u * 8 + 8 && l < L; ++l) {
        const uint32_t a = ivl[(l * N + n) * 2], b = ivl[(l * N + n) * 2 + 1];
        if (b < a) continue;
        lo = any ? (a < lo ? a : lo) : a;
        hi = any ? (b > hi ? b : hi) : b;
        any = true;
      }
      if (any) {
        t->unit_lo[n][u] = lo;
        t->unit_hi[n][u] = hi;
      }
      t->unit_width_sorted[n][u] = any ? hi - lo + 1 : 0;
    }
    std::sort(t->unit_width_sorted[n].begin(), t->unit_width_sorted[n].end());
  }
}

}  // namespace

extern "C" {

alto_status alto_options_init(alto_options* opt) {
  if (opt == nullptr) return fail(ALTO_EINVAL, "null options");
  std::memset(opt, 0, sizeof(*opt));
  opt->use_flags = 1;
  return ALTO_OK;
}

const char* alto_last_error(void) { return g_err; }

alto_status alto_create(alto_t* out, int nmodes, const uint64_t* dims, int64_t nnz,
                        const void* const* idx, int idx_bytes, const void* vals, alto_dtype vdtype,
                        const alto_options* opt, void* stream) {
  g_err[0] = '\0';
  if (out == nullptr || dims == nullptr) return fail(ALTO_EINVAL, "null output handle or dims");
  *out = nullptr;
  if (nnz < 0 || nnz >= (int64_t(1) << 32)) return fail(ALTO_EINVAL, "nnz %lld outside [0, 2^32)", (long long)nnz);
  if (nnz > 0 && (idx == nullptr || vals == nullptr)) return fail(ALTO_EINVAL, "null indices or values");
  if (idx_bytes != 4 && idx_bytes != 8) return fail(ALTO_EINVAL, "idx_bytes must be 4 or 8");
  if (vdtype != ALTO_F64 && vdtype != ALTO_F32 && vdtype != ALTO_BF16)
    return fail(ALTO_EINVAL, "values must be F64, F32 or BF16");
  alto_options o;
  alto_options_init(&o);
  if (opt != nullptr) o = *opt;
  if (o.nparts < 0) return fail(ALTO_EINVAL, "nparts must be >= 0");
  if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(ALTO_EINVAL, "alloc and free must both be set");
  Layout lay;
  alto_status st = make_layout(nmodes, dims, o.key_bits, &lay);
  if (st != ALTO_OK) return st;
  if (nnz > 0)
    for (int n = 0; n < nmodes; ++n)
      if (idx[n] == nullptr) return fail(ALTO_EINVAL, "index array %d is null", n);
  for (int n = 0; n < nmodes; ++n)
    if (o.variant[n] < ALTO_VAR_AUTO || o.variant[n] > ALTO_VAR_GENERIC)
      return fail(ALTO_EINVAL, "bad variant %d for mode %d", o.variant[n], n);

  alto_tensor_s* t = new (std::nothrow) alto_tensor_s();
  if (t == nullptr) return fail(ALTO_ENOMEM, "host allocation failed");
  t->alloc_fn = o.alloc;
  t->free_fn = o.free;
  t->alloc_ctx = o.ctx;
  t->M = nnz;
  t->vdtype = vdtype;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int N = nmodes;
  const int KW = lay.KW;
  const size_t vb = vdtype == ALTO_F64 ? 8 : (vdtype == ALTO_F32 ? 4 : 2);
  // temporaries
  std::vector<void*> staged;
  uint64_t* keys_alt = nullptr;
  uint32_t* perm_alt = nullptr;
  uint32_t* scratch = nullptr;
  uint32_t* first[kMaxModes] = {};
  uint32_t* last[kMaxModes] = {};
  uint32_t* cnt[kMaxModes] = {};
  uint32_t* hotbuf = nullptr;   // 2 * kHotCap (count, row) pairs + counter
  uint32_t* hotmap[kMaxModes] = {};
  unsigned long long* hist = nullptr;
  unsigned long long* dstat = nullptr;  // [0..N) distinct, [N..2N) max interval
  double* dnorm = nullptr;
  const void* dvals = vals;
  IdxPtrs ip{};
  int hstatus = 0;
  unsigned long long hstat[2 * kMaxModes] = {};
  int nflag = 0;
  std::vector<uint32_t> hivl;

  for (int n = 0; n < N; ++n) {
    t->reuse[n] = static_cast<double>(nnz) / static_cast<double>(lay.dims[n]);
    t->variant[n] = o.variant[n];
  }
  // helper flags go only into spare bits of the stored word (Sec. 3.3): they never widen it
  if (o.use_flags) {
    for (int n = 0; n < N; ++n)
      if (t->reuse[n] <= 4.0) ++nflag;
    if (nflag > 0 && lay.B + nflag <= 32 * lay.CW) {
      int b = lay.B;
      for (int n = 0; n < N; ++n)
        if (t->reuse[n] <= 4.0) lay.flag_bit[n] = b++;
    } else {
      nflag = 0;
    }
  }
  // hot-row flags for the buffered (reuse > 4) modes, in the bits left over
  int nhotbit = 0;
  if (o.use_flags) {
    int b = lay.B + nflag;
    for (int n = 0; n < N; ++n)
      if (t->reuse[n] > 4.0 && b < 32 * lay.CW && lay.dims[n] <= (1ull << 31)) {
        lay.hot_bit[n] = b++;
        ++nhotbit;
      }
  }
  t->lay = lay;
  t->L = nnz > 0 ? (o.nparts > 0 ? (o.nparts < nnz ? o.nparts : nnz) : auto_segments(nnz)) : 1;

  ALLOC(t->status, int*, sizeof(int) * 4);
  CK(cudaMemsetAsync(t->status, 0, sizeof(int) * 4, s));
  ALLOC(t->keys, uint64_t*, sizeof(uint64_t) * KW * (nnz + 32));
  ALLOC(t->perm, uint32_t*, sizeof(uint32_t) * (nnz + 32));
  ALLOC(t->vals, void*, vb * (nnz + 32));
  ALLOC(t->ivl, uint32_t*, sizeof(uint32_t) * 2 * N * t->L);
  ALLOC(dstat, unsigned long long*, sizeof(unsigned long long) * 2 * kMaxModes);
  ALLOC(dnorm, double*, sizeof(double));
  CK(cudaMemsetAsync(dstat, 0, sizeof(unsigned long long) * 2 * kMaxModes, s));
  CK(cudaMemsetAsync(dnorm, 0, sizeof(double), s));
  if (nnz > 0) {
    // stage host inputs on the device
    for (int n = 0; n < N; ++n) {
      if (is_device_ptr(idx[n])) {
        ip.p[n] = idx[n];
      } else {
        void* d = dev_alloc(t, static_cast<size_t>(nnz) * idx_bytes);
        if (d == nullptr) {
          st = fail(ALTO_ENOMEM, "staging allocation failed");
          goto done;
        }
        staged.push_back(d);
        CK(cudaMemcpyAsync(d, idx[n], static_cast<size_t>(nnz) * idx_bytes, cudaMemcpyHostToDevice, s));
        ip.p[n] = d;
      }
    }
    if (!is_device_ptr(vals)) {
      void* d = dev_alloc(t, static_cast<size_t>(nnz) * vb);
      if (d == nullptr) {
        st = fail(ALTO_ENOMEM, "staging allocation failed");
        goto done;
      }
      staged.push_back(d);
      CK(cudaMemcpyAsync(d, vals, static_cast<size_t>(nnz) * vb, cudaMemcpyHostToDevice, s));
      dvals = d;
    }
    ALLOC(keys_alt, uint64_t*, sizeof(uint64_t) * KW * (nnz + 32));
    ALLOC(perm_alt, uint32_t*, sizeof(uint32_t) * (nnz + 32));
    ALLOC(scratch, uint32_t*, sizeof(uint32_t) * sort_scratch_words(nnz));
    // 1. linearization
    CK(launch_encode(lay, ip, idx_bytes, nnz, t->keys, t->status, s));
    // 2. ordering
    CK(radix_sort_pairs(&t->keys, &keys_alt, &t->perm, &perm_alt, nnz, KW, lay.B, scratch, s));
    // 3. values into ALTO order
    CK(launch_permute(dvals, t->vals, t->perm, nnz, static_cast<int>(vb), s));
    CK(launch_sumsq(t->keys, KW, t->vals, vdtype, nnz, dnorm, s));
    // 4-5. partitioning, intervals, per-row first/last segment
    for (int n = 0; n < N; ++n) {
      ALLOC(first[n], uint32_t*, sizeof(uint32_t) * lay.dims[n]);
      CK(cudaMemsetAsync(first[n], 0xff, sizeof(uint32_t) * lay.dims[n], s));
      ALLOC(cnt[n], uint32_t*, sizeof(uint32_t) * lay.dims[n]);
      CK(cudaMemsetAsync(cnt[n], 0, sizeof(uint32_t) * lay.dims[n], s));
      if (lay.flag_bit[n] >= 0) {
        ALLOC(last[n], uint32_t*, sizeof(uint32_t) * lay.dims[n]);
        CK(cudaMemsetAsync(last[n], 0, sizeof(uint32_t) * lay.dims[n], s));
      }
    }
    CK(launch_segment_stats(lay, t->keys, nnz, t->L, t->ivl, first, last, cnt, s));
    // hot rows per mode: threshold on the sampled counts, hottest first
    ALLOC(hist, unsigned long long*, sizeof(unsigned long long) * 33);
    ALLOC(hotbuf, uint32_t*, sizeof(uint32_t) * (2 * kHotCap + 1));
    for (int n = 0; n < N; ++n) {
      unsigned long long hh[33] = {};
      CK(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 33, s));
      CK(launch_hot_hist(cnt[n], lay.dims[n], hist, s));
      CK(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      int b = 1;
      unsigned long long above = 0;
      for (int k = 1; k < 33; ++k) above += hh[k];
      while (b < 33 && above > static_cast<unsigned long long>(kHotCap)) above -= hh[b++];
      if (b >= 33 || above == 0) continue;
      CK(cudaMemsetAsync(hotbuf + 2 * kHotCap, 0, sizeof(uint32_t), s));
      CK(launch_hot_collect(cnt[n], lay.dims[n], 1u << b, kHotCap, hotbuf, hotbuf + 2 * kHotCap, s));
      std::vector<uint32_t> h(2 * kHotCap + 1);
      CK(cudaMemcpyAsync(h.data(), hotbuf, sizeof(uint32_t) * h.size(), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      int nh = static_cast<int>(h[2 * kHotCap] < static_cast<uint32_t>(kHotCap) ? h[2 * kHotCap] : kHotCap);
      std::vector<std::pair<uint32_t, uint32_t>> pr(nh);
      for (int k = 0; k < nh; ++k) pr[k] = {h[2 * k], h[2 * k + 1]};
      std::sort(pr.begin(), pr.end(), [](const std::pair<uint32_t, uint32_t>& x,
                                         const std::pair<uint32_t, uint32_t>& y) {
        return x.first != y.first ? x.first > y.first : x.second < y.second;
      });
      std::vector<uint32_t> rows;
      double hot_samples = 0.0;
      for (int k = 0; k < nh; ++k)
        if (pr[k].second != 0xffffffffu) {  // that value marks empty slots
          rows.push_back(pr[k].second);
          hot_samples += pr[k].first;
        }
      nh = static_cast<int>(rows.size());
      t->hot_share[n] = hot_samples / static_cast<double>((nnz + kHotSample - 1) / kHotSample);
      ALLOC(t->hot[n], uint32_t*, sizeof(uint32_t) * (nh > 0 ? nh : 1));
      CK(cudaMemcpyAsync(t->hot[n], rows.data(), sizeof(uint32_t) * nh, cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
      t->hot_n[n] = nh;
      if (lay.hot_bit[n] >= 0 && nh > 0) {
        const size_t words = (lay.dims[n] + 31) / 32;
        ALLOC(hotmap[n], uint32_t*, sizeof(uint32_t) * words);
        CK(cudaMemsetAsync(hotmap[n], 0, sizeof(uint32_t) * words, s));
        CK(launch_hot_map(t->hot[n], nh, hotmap[n], s));
      }
    }
    for (int n = 0; n < N; ++n) CK(launch_count_touched(first[n], lay.dims[n], dstat + n, s));
    CK(launch_max_interval(t->ivl, t->L, N, dstat + kMaxModes, s));
    if (nflag > 0) CK(launch_set_flags(lay, t->keys, nnz, first, last, nullptr, s));
    if (nhotbit > 0) CK(launch_set_flags(lay, t->keys, nnz, first, last, hotmap, s));
    // stored keys: packed into CW 32-bit words when that is narrower
    if (lay.CW < 2 * KW) {
      ALLOC(t->ckeys, uint32_t*, sizeof(uint32_t) * lay.CW * (nnz + 32));
      CK(launch_pack_keys(t->keys, KW, t->ckeys, lay.CW, nnz, s));
    }
  } else {
    // empty tensor: one empty segment
    std::vector<uint32_t> e(2 * N);
    for (int n = 0; n < N; ++n) {
      e[2 * n] = 1;
      e[2 * n + 1] = 0;
    }
    CK(cudaMemcpyAsync(t->ivl, e.data(), sizeof(uint32_t) * 2 * N, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(hstat, dstat, sizeof(hstat), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&t->normX2, dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hstatus, t->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  hivl.resize(static_cast<size_t>(2) * N * t->L);
  CK(cudaMemcpyAsync(hivl.data(), t->ivl, sizeof(uint32_t) * hivl.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hstatus != 0) {
    st = fail(static_cast<alto_status>(hstatus),
              hstatus == ALTO_ERANGE ? "an input index is >= its mode length" : "device error %d", hstatus);
    goto done;
  }
  for (int n = 0; n < N; ++n) {
    t->distinct[n] = hstat[n];
    t->max_ivl[n] = hstat[kMaxModes + n];
  }
  unit_intervals(t, hivl);
  if (t->ckeys != nullptr) {  // packed: the generation-width keys are no longer needed
    dev_free(t, t->keys);
    t->keys = nullptr;
  } else {
    t->ckeys = reinterpret_cast<uint32_t*>(t->keys);
  }
  st = ALTO_OK;

done:
  cudaStreamSynchronize(s);  // temporaries may still be in use on failure
  for (void* p : staged) dev_free(t, p);
  dev_free(t, keys_alt);
  dev_free(t, perm_alt);
  dev_free(t, scratch);
  for (int n = 0; n < kMaxModes; ++n) {
    dev_free(t, first[n]);
    dev_free(t, last[n]);
    dev_free(t, cnt[n]);
    dev_free(t, hotmap[n]);
  }
  dev_free(t, hotbuf);
  dev_free(t, hist);
  dev_free(t, dstat);
  dev_free(t, dnorm);
  if (st != ALTO_OK) {
    free_format(t);
    delete t;
    return st;
  }
  *out = t;
  return ALTO_OK;
}

alto_status alto_mttkrp(alto_t t, int mode, const void* const* factors, int rank, alto_dtype fdtype,
                        void* out, void* stream) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  return run_mttkrp(t, mode, factors, rank, fdtype, out, ALTO_VAR_AUTO, static_cast<cudaStream_t>(stream));
}

alto_status alto_cpals(alto_t t, int rank, int iters, void* const* factors, alto_dtype fdtype, double* lambda,
                       double* fit, void* stream) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  alto_status st = run_cpals(t, rank, iters, factors, fdtype, lambda, fit, s);
  if (st != ALTO_OK) return st;
  if (fit != nullptr) return alto_check(t, stream);
  return ALTO_OK;
}

alto_status alto_get_layout(alto_t t, int* nmodes, int* bits_per_mode, uint64_t* masks, int* key_words,
                            int* flag_bit, int* hot_bit) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  const Layout& L = t->lay;
  if (nmodes) *nmodes = L.N;
  if (key_words) *key_words = L.KW;
  for (int n = 0; n < L.N; ++n) {
    if (bits_per_mode) bits_per_mode[n] = L.nbits[n];
    if (masks) {
      masks[2 * n] = L.mask[n][0];
      masks[2 * n + 1] = L.mask[n][1];
    }
    if (flag_bit) flag_bit[n] = L.flag_bit[n];
    if (hot_bit) hot_bit[n] = L.hot_bit[n];
  }
  return ALTO_OK;
}

alto_status alto_get_stats(alto_t t, int64_t* nnz, int64_t* nparts, uint64_t* distinct, double* reuse,
                           int* variant, uint64_t* max_interval) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  if (nnz) *nnz = t->M;
  if (nparts) *nparts = t->L;
  for (int n = 0; n < t->lay.N; ++n) {
    if (distinct) distinct[n] = t->distinct[n];
    if (reuse) reuse[n] = t->reuse[n];
    if (variant) variant[n] = t->variant[n];
    if (max_interval) max_interval[n] = t->max_ivl[n];
  }
  return ALTO_OK;
}

alto_status alto_export(alto_t t, uint64_t* keys, uint32_t* perm, void* vals, int64_t* bounds,
                        uint32_t* intervals) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  alto_status st = ALTO_OK;
  const size_t M = static_cast<size_t>(t->M);
  const size_t vb = t->vdtype == ALTO_F64 ? 8 : (t->vdtype == ALTO_F32 ? 4 : 2);
  if (keys && M) {  // stored keys widened to KW 64-bit words
    const int CW = t->lay.CW, KW = t->lay.KW;
    std::vector<uint32_t> h(static_cast<size_t>(CW) * M);
    CK(cudaMemcpy(h.data(), t->ckeys, sizeof(uint32_t) * h.size(), cudaMemcpyDeviceToHost));
    for (size_t x = 0; x < M; ++x)
      for (int w = 0; w < KW; ++w) {
        const uint64_t lo = 2 * w < CW ? h[x * CW + 2 * w] : 0u;
        const uint64_t hi = 2 * w + 1 < CW ? h[x * CW + 2 * w + 1] : 0u;
        keys[x * KW + w] = lo | (hi << 32);
      }
  }
  if (perm && M) CK(cudaMemcpy(perm, t->perm, sizeof(uint32_t) * M, cudaMemcpyDeviceToHost));
  if (vals && M) CK(cudaMemcpy(vals, t->vals, vb * M, cudaMemcpyDeviceToHost));
  if (intervals)
    CK(cudaMemcpy(intervals, t->ivl, sizeof(uint32_t) * 2 * t->lay.N * t->L, cudaMemcpyDeviceToHost));
  if (bounds)
    for (int64_t l = 0; l <= t->L; ++l) bounds[l] = seg_begin(l, t->M, t->L);
done:
  return st;
}

alto_status alto_get_hot_rows(alto_t t, int mode, uint32_t* rows, int* count) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  if (mode < 0 || mode >= t->lay.N) return fail(ALTO_EINVAL, "bad mode %d", mode);
  if (count) *count = t->hot_n[mode];
  if (rows && t->hot_n[mode] > 0) {
    const cudaError_t e =
        cudaMemcpy(rows, t->hot[mode], sizeof(uint32_t) * t->hot_n[mode], cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(ALTO_ECUDA, "hot rows: %s", cudaGetErrorString(e));
  }
  return ALTO_OK;
}

alto_status alto_get_mode_stats(alto_t t, int mode, double* out, int n) {
  if (t == nullptr || out == nullptr) return fail(ALTO_EINVAL, "null argument");
  if (mode < 0 || mode >= t->lay.N) return fail(ALTO_EINVAL, "bad mode %d", mode);
  const std::vector<uint32_t>& w = t->unit_width_sorted[mode];
  const double med = w.empty() ? 0.0 : static_cast<double>(w[w.size() / 2]);
  const double p90 = w.empty() ? 0.0 : static_cast<double>(w[(w.size() * 9) / 10]);
  const double v[8] = {static_cast<double>(t->lay.dims[mode]), static_cast<double>(t->distinct[mode]), t->reuse[mode],
                       static_cast<double>(t->max_ivl[mode]), static_cast<double>(t->hot_n[mode]), t->hot_share[mode],
                       med, p90};
  for (int i = 0; i < n && i < 8; ++i) out[i] = v[i];
  for (int i = 8; i < n; ++i) out[i] = 0.0;
  return ALTO_OK;
}

alto_status alto_get_unit_fit(alto_t t, int mode, uint64_t rows, double* frac) {
  if (t == nullptr || frac == nullptr) return fail(ALTO_EINVAL, "null argument");
  if (mode < 0 || mode >= t->lay.N) return fail(ALTO_EINVAL, "bad mode %d", mode);
  *frac = t->unit_fit_frac(mode, rows);
  return ALTO_OK;
}

alto_status alto_set_variant(alto_t t, int mode, int variant) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  if (mode < 0 || mode >= t->lay.N) return fail(ALTO_EINVAL, "bad mode %d", mode);
  if (variant < ALTO_VAR_AUTO || variant > ALTO_VAR_GENERIC) return fail(ALTO_EINVAL, "bad variant %d", variant);
  t->variant[mode] = variant;
  return ALTO_OK;
}

alto_status alto_set_gram_engine(alto_t t, int engine) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  if (engine < ALTO_GRAM_AUTO || engine > ALTO_GRAM_TENSOR_CORES) return fail(ALTO_EINVAL, "bad engine %d", engine);
  t->gram_engine = engine;
  return ALTO_OK;
}

alto_status alto_gram(const void* U, int64_t I, int R, alto_dtype dtype, int engine, double* G, void* stream) {
  return gram_any(U, I, R, dtype, engine, G, static_cast<cudaStream_t>(stream));
}

alto_status alto_set_parts(alto_t t, int mode, int64_t nparts) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  if (mode < 0 || mode >= t->lay.N) return fail(ALTO_EINVAL, "bad mode %d", mode);
  if (nparts < 0) return fail(ALTO_EINVAL, "negative segment count %lld", static_cast<long long>(nparts));
  t->mode_parts[mode] = nparts;
  return ALTO_OK;
}

alto_status alto_get_key_bytes(alto_t t, int* bytes) {
  if (t == nullptr || bytes == nullptr) return fail(ALTO_EINVAL, "null argument");
  *bytes = 4 * t->lay.CW;
  return ALTO_OK;
}

alto_status alto_check(alto_t t, void* stream) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  alto_status st = ALTO_OK;
  int h = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(&h, t->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    CK(cudaMemset(t->status, 0, sizeof(int)));
    return fail(static_cast<alto_status>(h), "device reported status %d", h);
  }
done:
  return st;
}

alto_status alto_profile(alto_t t, int enable) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  t->prof = enable != 0;
  return ALTO_OK;
}

alto_status alto_profile_read(alto_t t, double* ms, int64_t* calls) {
  if (t == nullptr) return fail(ALTO_EINVAL, "null tensor");
  const int N = t->lay.N;
  for (int n = 0; n < N; ++n) {
    if (ms) ms[n] = 0.0;
    if (calls) calls[n] = 0;
  }
  for (size_t i = 0; i < t->ev_used; ++i) {
    cudaError_t e = cudaEventSynchronize(t->ev_pool[2 * i + 1]);
    float f = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, t->ev_pool[2 * i], t->ev_pool[2 * i + 1]);
    if (e != cudaSuccess) {
      t->ev_used = 0;
      return fail(ALTO_ECUDA, "profile read: %s", cudaGetErrorString(e));
    }
    const int m = t->ev_mode[i];
    if (ms) ms[m] += f;
    if (calls) calls[m] += 1;
  }
  t->ev_used = 0;
  return ALTO_OK;
}

alto_status alto_launch_count(uint64_t* count) {
  if (count == nullptr) return fail(ALTO_EINVAL, "null count");
  *count = g_launches.load(std::memory_order_relaxed);
  return ALTO_OK;
}

alto_status alto_destroy(alto_t t) {
  if (t == nullptr) return ALTO_OK;
  free_format(t);
  delete t;
  return ALTO_OK;
}

alto_status alto_layout_for_dims(int nmodes, const uint64_t* dims, int key_bits, int* bits_per_mode,
                                 uint64_t* masks, int* key_words, int* total_bits) {
  if (dims == nullptr) return fail(ALTO_EINVAL, "null dims");
  Layout L;
  const alto_status st = make_layout(nmodes, dims, key_bits, &L);
  if (st != ALTO_OK) return st;
  for (int n = 0; n < L.N; ++n) {
    if (bits_per_mode) bits_per_mode[n] = L.nbits[n];
    if (masks) {
      masks[2 * n] = L.mask[n][0];
      masks[2 * n + 1] = L.mask[n][1];
    }
  }
  if (key_words) *key_words = L.KW;
  if (total_bits) *total_bits = L.B;
  return ALTO_OK;
}

alto_status alto_decode_host(int nmodes, const uint64_t* dims, int key_bits, int64_t count,
                             const uint64_t* keys, uint32_t* idx) {
  if (dims == nullptr || (count > 0 && (keys == nullptr || idx == nullptr)))
    return fail(ALTO_EINVAL, "null argument");
  Layout L;
  const alto_status st = make_layout(nmodes, dims, key_bits, &L);
  if (st != ALTO_OK) return st;
  for (int64_t x = 0; x < count; ++x) {
    uint64_t k[2] = {keys[x * L.KW], L.KW == 2 ? keys[x * L.KW + 1] : 0};
    host_decode(L, k, idx + x * L.N);
  }
  return ALTO_OK;
}

}  // extern "C"
