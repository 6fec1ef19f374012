// Gram matrix G = U^T U of a BF16 factor (I x R, row-major, R in {8, 16, 32,
// 64}) on the 5th-generation tensor cores -- the one dense contraction of a
// CP-ALS iteration (Sec. 2.2: V is the Hadamard product of the other modes'
// Gram matrices).  BF16 x BF16 products are exact in FP32, the tensor core
// sums them in FP32 per thread block, and the blocks' partials are added in
// FP64 -- the precision split of the CUDA-core Gram.
//
// Per block (128 threads, 4 warps): rows of U are taken 64 at a time (the K
// dimension of the product).  The block writes the chunk into shared memory
// transposed, as a K-major tile of 128 "rows" (the M dimension, rows >= R are
// never read back) x 64 k, in the canonical no-swizzle layout: 8 x 8 core
// matrices of 128 contiguous bytes (8 rows x 16 bytes), K-adjacent core
// matrices 128 bytes apart (leading byte offset), row-adjacent ones 1024
// bytes apart (stride byte offset).  One elected thread issues four
// tcgen05.mma kind::f16 (M = 128, N = max(R, 16), K = 16 each) with A and B
// both read from that tile -- D[m][n] = sum_k U[k][m] U[k][n] -- accumulating
// into tensor memory, and commits them to an mbarrier.  Two tiles alternate,
// so the next chunk is loaded and transposed while the tensor core works.
// Every 16 chunks (1024 rows) and at the end, warps 0..R/32 read their 32
// accumulator lanes (tcgen05.ld) into FP64 sums in shared memory and the
// accumulator restarts, so no FP32 sum runs over more than 1024 products; the
// block's FP64 sums go into the Gram with atomics.
//
// NORM form (CP-ALS with BF16 factors): the chunk is read from the solved FP32
// rows A instead, divided by lambda, rounded to BF16, stored as U and staged
// in the same step; optionally it adds the fit's inner product
// sum_r lambda_r sum_i U[i,r] Mt[i,r].
//
// Every mbarrier wait is bounded; a wait that runs out records ALTO_ETIMEOUT
// in the status word, skips the rest, waits (bounded) for the block's last
// commit and frees the tensor memory before returning.
#include "internal.h"

namespace alto {

namespace {

constexpr int kGT = 128;               // threads per block
constexpr int kGK = 64;                // rows of U per chunk (K)
constexpr int kTileBytes = 128 * kGK * 2;  // 128 M-rows x 64 k, BF16
constexpr int kLBO = 128;              // K-adjacent core matrices
constexpr int kSBO = 1024;             // M-adjacent core matrices (8 per chunk along K)
constexpr uint32_t kSpin = 1u << 22;   // try_wait rounds before giving up
constexpr int kFlushChunks = 16;       // chunks (1024 rows) summed in FP32 before an FP64 flush

struct GramTcArgs {
  const void* src;   // BF16 U (plain) or FP32 A (NORM), I x R
  int64_t I;
  int R;
  double* G;         // R x R, FP64, accumulated into
  int* status;
  // NORM only
  const double* colstat;
  int use_max;
  double* lambda;
  __nv_bfloat16* U;
  const float* Mt;
  double* ip;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((kLBO >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((kSBO >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// byte offset of element (m, k) of the K-major tile
__device__ __forceinline__ int tile_off(int m, int k) {
  return (m >> 3) * kSBO + (k >> 3) * kLBO + (m & 7) * 16 + (k & 7) * 2;
}

// Warps 0..R/32: add accumulator rows m < R (tensor-memory lane m, columns
// 0..R-1) into the FP64 sums gacc (each thread owns its row: no conflicts).
__device__ __forceinline__ void flush_accumulator(uint32_t tmem, int R, double* gacc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp * 32 >= R) return;
  const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  const int m = warp * 32 + lane;
  for (int c0 = 0; c0 < R; c0 += 8) {
    uint32_t v[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "r"(taddr + static_cast<uint32_t>(c0))
        : "memory");
    if (m < R) {
#pragma unroll
      for (int e = 0; e < 8; ++e) gacc[m * R + c0 + e] += static_cast<double>(__uint_as_float(v[e]));
    }
  }
}

template <bool NORM>
__global__ void __launch_bounds__(kGT) gram_tc_kernel(const __grid_constant__ GramTcArgs g) {
  __shared__ __align__(1024) uint8_t tile[2][kTileBytes];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float inv[64];
  __shared__ double lam[64];
  __shared__ double ipred[kGT / 32];
  extern __shared__ double gacc[];  // R x R FP64 sums (dynamic: R * R * 8 bytes)
  const int R = g.R;
  const int N = R < 16 ? 16 : R;
  const uint32_t ncols = N <= 32 ? 32u : 64u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (NORM) {
    for (int r = threadIdx.x; r < R; r += kGT) {
      const double l = g.use_max ? fmax(g.colstat[r], 1.0) : sqrt(g.colstat[r]);
      lam[r] = l;
      inv[r] = static_cast<float>(1.0 / l);
      if (blockIdx.x == 0) g.lambda[r] = l;
    }
  }
  // rows m >= R of the tiles feed only accumulator rows that are never read;
  // zero them once so that they hold finite values
  for (int i = threadIdx.x; i < 2 * kTileBytes / 16; i += kGT)
    reinterpret_cast<uint4*>(&tile[0][0])[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = threadIdx.x; i < R * R; i += kGT) gacc[i] = 0.0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = mma_idesc(128, N);

  const int CG = R / 8;                  // 8-column groups of a row
  const int groups = kGK * CG;           // per chunk
  const int64_t nchunks = (g.I + kGK - 1) / kGK;
  double ipd = 0.0;
  bool ok = true;
  int it = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++it) {
    const int buf = it & 1;
    const int64_t k0 = ch * kGK;
    if (it > 0 && it % kFlushChunks == 0) {
      // every MMA so far has completed once the last commit has: move the
      // FP32 accumulator into the FP64 sums and start it again
      if (!mbar_wait(smem_u32(&mbar[(it - 1) & 1]), ((it - 1) >> 1) & 1)) ok = false;
      if (!__syncthreads_and(ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      flush_accumulator(tmem, R, gacc);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    // load (and, for NORM, normalise, round and store) this thread's groups
    uint4 vals[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = threadIdx.x + q * kGT;
      vals[q] = make_uint4(0u, 0u, 0u, 0u);
      if (gi >= groups) continue;
      const int k = gi / CG, c = (gi - k * CG) * 8;
      const int64_t row = k0 + k;
      if (row >= g.I) continue;
      if constexpr (NORM) {
        const float* a = static_cast<const float*>(g.src) + row * R + c;
        const float4 x0 = *reinterpret_cast<const float4*>(a);
        const float4 x1 = *reinterpret_cast<const float4*>(a + 4);
        const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        __nv_bfloat16 h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(xs[e] * inv[c + e]);
        vals[q] = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(g.U + row * R + c) = vals[q];
        if (g.Mt != nullptr) {
          const float* mt = g.Mt + row * R + c;
#pragma unroll
          for (int e = 0; e < 8; ++e)
            ipd += static_cast<double>(__bfloat162float(h[e]) * mt[e]) * lam[c + e];
        }
      } else {
        vals[q] = __ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(g.src) + row * R + c));
      }
    }
    // the tile is free once the MMAs of two chunks ago have completed
    if (it >= 2 && !mbar_wait(smem_u32(&mbar[buf]), ((it - 2) >> 1) & 1)) ok = false;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    uint8_t* t = tile[buf];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = threadIdx.x + q * kGT;
      if (gi >= groups) continue;
      const int k = gi / CG, c = (gi - k * CG) * 8;
      const uint16_t* h = reinterpret_cast<const uint16_t*>(&vals[q]);
#pragma unroll
      for (int e = 0; e < 8; ++e) *reinterpret_cast<uint16_t*>(t + tile_off(c + e, k)) = h[e];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(t);
#pragma unroll
      for (int j = 0; j < kGK / 16; ++j) {
        const uint64_t d = smem_desc(base + j * 2 * kLBO);
        const uint32_t acc = (it % kFlushChunks > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(d), "l"(d), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[buf]))
                   : "memory");
    }
  }
  // the last commit covers every MMA of the block
  bool drained = true;
  if (it > 0) drained = mbar_wait(smem_u32(&mbar[(it - 1) & 1]), ((it - 1) >> 1) & 1);
  const bool good = __syncthreads_and(ok && drained);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // the chunks since the last flush (at least one whenever it > 0)
  if (good && it > 0) flush_accumulator(tmem, R, gacc);
  __syncthreads();
  if (good && it > 0)
    for (int e = threadIdx.x; e < R * R; e += kGT) atomicAdd(g.G + e, gacc[e]);
  if (!good && threadIdx.x == 0 && g.status != nullptr) atomicCAS(g.status, 0, static_cast<int>(ALTO_ETIMEOUT));
  if constexpr (NORM) {
    if (g.Mt != nullptr) {
      for (int o = 16; o > 0; o >>= 1) ipd += __shfl_xor_sync(0xffffffffu, ipd, o);
      if (lane == 0) ipred[warp] = ipd;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (NORM) {
    if (g.Mt != nullptr && threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kGT / 32; ++w) s += ipred[w];
      atomicAdd(g.ip, s);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

unsigned gram_tc_grid(int64_t I) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int64_t g = (I + kGK - 1) / kGK;
  const int64_t cap = static_cast<int64_t>(sms) * 3;  // up to 3 blocks of ~66 KB shared memory per SM
  if (g > cap) g = cap;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

}  // namespace

bool gram_tc_supported(int R) { return R == 8 || R == 16 || R == 32 || R == 64; }

cudaError_t launch_gram_bf16_tc(const __nv_bfloat16* U, int64_t I, int R, double* G, int* status,
                                cudaStream_t s) {
  if (I <= 0) return cudaSuccess;
  GramTcArgs a{};
  a.src = U;
  a.I = I;
  a.R = R;
  a.G = G;
  a.status = status;
  const size_t dyn = sizeof(double) * R * R;
  cudaFuncSetAttribute(gram_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
  gram_tc_kernel<false><<<gram_tc_grid(I), kGT, dyn, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_normalize_gram_bf16_tc(const float* A, int64_t I, int R, const double* colstat, int use_max,
                                          double* lambda, __nv_bfloat16* U, double* G, const float* Mt,
                                          double* ip, int* status, cudaStream_t s) {
  GramTcArgs a{};
  a.src = A;
  a.I = I;
  a.R = R;
  a.G = G;
  a.status = status;
  a.colstat = colstat;
  a.use_max = use_max;
  a.lambda = lambda;
  a.U = U;
  a.Mt = Mt;
  a.ip = ip;
  const size_t dyn = sizeof(double) * R * R;
  cudaFuncSetAttribute(gram_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
  gram_tc_kernel<true><<<gram_tc_grid(I), kGT, dyn, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace alto
