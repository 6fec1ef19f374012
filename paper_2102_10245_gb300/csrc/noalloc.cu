// alto_linearize_noalloc: ALTO linearization and ordering into caller
// buffers, with every scratch buffer in one fixed, file-scope device array,
// so the call never allocates device memory.
//
// Some callers cannot allocate: services that reserve all device memory for
// their own pool up front, and embedders whose device allocator belongs to
// another runtime (a cudaMalloc behind its back would break its accounting).
// They still pass their own inputs and outputs; this entry point supplies the
// sort's scratch itself.  The call reads its status word back and
// synchronises the stream before it returns.
//
// The array is kScratchWords 8-byte words (about 5.3 MB) of device memory
// that every GPU which loads
// libalto keeps until the process exits.  All calls share it: two calls whose
// work overlaps on the GPU (different streams, or different host threads on
// one device) race on it and must be serialised by the caller.
#include "internal.h"

namespace alto {

namespace {

constexpr int64_t kNoAllocMaxNnz = ALTO_NOALLOC_MAX_NNZ;
// scratch layout, in 8-byte words: alternate keys (2 words per nonzero),
// alternate positions (uint32), sort counts / offsets / scan partials
// (uint32), and the status word
constexpr size_t kKeyAltWords = 2 * static_cast<size_t>(kNoAllocMaxNnz);
constexpr size_t kPermAltWords = static_cast<size_t>(kNoAllocMaxNnz) / 2;
constexpr size_t kSortWords = (static_cast<size_t>(sort_scratch_words_for(kNoAllocMaxNnz)) + 1) / 2;
constexpr size_t kStatusWords = 4;
constexpr size_t kScratchWords = kKeyAltWords + kPermAltWords + kSortWords + kStatusWords;

__device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

// Device address of the scratch array in the current context.  The array's
// name in host code only stands in for the symbol; the address is looked up
// on every call (cheap once the module is loaded), so a context that was torn
// down and re-created (cudaDeviceReset) gets the new array, not a stale one.
alto_status scratch_for_current_device(unsigned long long** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  *out = static_cast<unsigned long long*>(p);
  return ALTO_OK;
}

}  // namespace

}  // namespace alto

using namespace alto;

extern "C" alto_status alto_linearize_noalloc(int nmodes, const uint64_t* dims, int64_t nnz,
                                              const void* const* idx, int idx_bytes, uint64_t* keys,
                                              uint32_t* perm, void* stream) {
  if (dims == nullptr) return fail(ALTO_EINVAL, "null dims");
  if (nnz < 0 || nnz > kNoAllocMaxNnz)
    return fail(ALTO_EINVAL, "nnz %lld outside [0, %lld] (the fixed scratch limit)", (long long)nnz,
                (long long)kNoAllocMaxNnz);
  if (idx_bytes != 4 && idx_bytes != 8) return fail(ALTO_EINVAL, "idx_bytes must be 4 or 8");
  Layout lay;
  alto_status st = make_layout(nmodes, dims, 0, &lay);
  if (st != ALTO_OK) return st;
  if (nnz == 0) return ALTO_OK;
  if (idx == nullptr || keys == nullptr || perm == nullptr) return fail(ALTO_EINVAL, "null buffer");
  IdxPtrs ip{};
  for (int n = 0; n < nmodes; ++n) {
    if (idx[n] == nullptr) return fail(ALTO_EINVAL, "index array %d is null", n);
    ip.p[n] = idx[n];
  }
  unsigned long long* base = nullptr;
  st = scratch_for_current_device(&base);
  if (st != ALTO_OK) return st;
  uint64_t* key_alt = reinterpret_cast<uint64_t*>(base);
  uint32_t* perm_alt = reinterpret_cast<uint32_t*>(base + kKeyAltWords);
  uint32_t* sort_scratch = reinterpret_cast<uint32_t*>(base + kKeyAltWords + kPermAltWords);
  int* status = reinterpret_cast<int*>(base + kKeyAltWords + kPermAltWords + kSortWords);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The sort ping-pongs between two buffers; start in the scratch one when the
  // pass count is odd so that the result lands in the caller's buffers.
  const int passes = sort_passes_for(lay.B);
  uint64_t* k0 = (passes & 1) ? key_alt : keys;
  uint64_t* k1 = (passes & 1) ? keys : key_alt;
  uint32_t* p0 = (passes & 1) ? perm_alt : perm;
  uint32_t* p1 = (passes & 1) ? perm : perm_alt;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_encode(lay, ip, idx_bytes, nnz, k0, status, s);
  if (e == cudaSuccess) e = radix_sort_pairs(&k0, &k1, &p0, &p1, nnz, lay.KW, lay.B, sort_scratch, s);
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "linearize: %s", cudaGetErrorString(e));
  if (k0 != keys || p0 != perm) return fail(ALTO_ECUDA, "linearize: result not in the caller's buffers");
  int h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "linearize: %s", cudaGetErrorString(e));
  if (h != 0) return fail(static_cast<alto_status>(h), "an input index is >= its mode length");
  return ALTO_OK;
}
