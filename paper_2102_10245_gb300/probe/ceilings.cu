// Hardware ceilings of the MTTKRP data path on this GPU (measured, not
// modelled):
//   gather2  -- every "nonzero" gathers two rows of a table (128-byte FP32
//               rank-32 rows or 64-byte BF16 rows) by random row index, with
//               the lane layout of the kernels (16 bytes per lane) and a
//               32-byte variant; table sizes from L1-resident to HBM-resident
//               give rows per clock per SM from each level of the hierarchy;
//   red_rows -- 128-byte rows added into random output rows with
//               red.global.add.v4.f32 (8 lanes per row), output sizes from a
//               contended hot set to HBM-resident;
//   decode3  -- the five-step parallel-suffix compress (Hacker's Delight,
//               2nd ed., Sec. 7-4) of three modes from 64-bit keys with the
//               4M x 4M x 30k layout, against a plain key stream.
// Indices are drawn by a splitmix64 hash modulo the table size, so every
// access stays inside its buffer.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e_), __LINE__); return 1; } } while (0)

__device__ __forceinline__ uint64_t mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull; x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull; return x ^ (x >> 31);
}
__global__ void fill_idx(uint32_t* idx, int64_t n, uint32_t T, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    idx[i] = (uint32_t)(mix(i ^ seed) % T);
}
__global__ void fill_f(float* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 1.0f + (float)(i & 7) * 0.125f;
}
__global__ void fill_k(uint64_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = mix(i) & ((1ull << 59) - 1);
}

template <int BYTES> struct Piece;
template <> struct Piece<8> { uint32_t w[2]; };
template <> struct Piece<16> { uint32_t w[4]; };
template <> struct Piece<32> { uint32_t w[8]; };

template <int BYTES>
__device__ __forceinline__ Piece<BYTES> ldp(const char* p) {
  Piece<BYTES> r;
  if constexpr (BYTES == 8) {
    uint2 a = __ldg(reinterpret_cast<const uint2*>(p)); r.w[0] = a.x; r.w[1] = a.y;
  } else if constexpr (BYTES == 16) {
    uint4 a = __ldg(reinterpret_cast<const uint4*>(p)); r.w[0] = a.x; r.w[1] = a.y; r.w[2] = a.z; r.w[3] = a.w;
  } else {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4]), "=r"(r.w[5]),
                   "=r"(r.w[6]), "=r"(r.w[7]) : "l"(p));
  }
  return r;
}

// each nonzero q gathers rows idx[2q], idx[2q+1] (ROWB bytes each) and
// accumulates their elementwise product (as fp32 words)
template <int ROWB, int PB>
__global__ void __launch_bounds__(256) gather2(const char* __restrict__ T, const uint32_t* __restrict__ idx,
                                               int64_t nq, float* out) {
  constexpr int LPR = ROWB / PB;      // lanes per row
  constexpr int NPI = 32 / LPR;       // nonzeros per instruction
  constexpr int W = PB / 4;
  const int lane = threadIdx.x & 31, g = lane / LPR, c = lane % LPR;
  const int64_t warps = (int64_t)gridDim.x * 8;
  float acc[W];
#pragma unroll
  for (int e = 0; e < W; ++e) acc[e] = 0.f;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32; base < nq; base += warps * 32) {
    uint2 ij = make_uint2(0, 0);
    if (base + lane < nq) ij = reinterpret_cast<const uint2*>(idx)[base + lane];
#pragma unroll
    for (int p = 0; p < 32 / NPI; ++p) {
      const int q = p * NPI + g;
      const uint32_t a = __shfl_sync(0xffffffffu, ij.x, q), b = __shfl_sync(0xffffffffu, ij.y, q);
      const Piece<PB> x = ldp<PB>(T + (size_t)a * ROWB + c * PB);
      const Piece<PB> y = ldp<PB>(T + (size_t)b * ROWB + c * PB);
#pragma unroll
      for (int e = 0; e < W; ++e) acc[e] = fmaf(__uint_as_float(x.w[e]), __uint_as_float(y.w[e]), acc[e]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int e = 0; e < W; ++e) s += acc[e];
  out[blockIdx.x * 256 + threadIdx.x] = s;
}

// every nonzero q adds a 128-B row into out row idx[q] with RED.v4 (8 lanes)
__global__ void __launch_bounds__(256) red_rows(float* out, const uint32_t* __restrict__ idx, int64_t nq) {
  const int lane = threadIdx.x & 31, g = lane / 8, c = lane % 8;
  const int64_t warps = (int64_t)gridDim.x * 8;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32; base < nq; base += warps * 32) {
    uint32_t r = 0;
    if (base + lane < nq) r = idx[base + lane];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const uint32_t row = __shfl_sync(0xffffffffu, r, p * 4 + g);
      float* a = out + (size_t)row * 32 + c * 4;
      asm volatile("red.global.add.v4.f32 [%0], {%1, %1, %1, %1};" ::"l"(a), "f"(1.0f) : "memory");
    }
  }
}

struct Dp { uint32_t mask[3][2]; uint32_t mv[3][2][5]; uint32_t shift[3][2]; };
// decode three modes from 2 key words, xor into a checksum
template <int DEC>
__global__ void __launch_bounds__(256) decode3(const uint64_t* __restrict__ keys, int64_t n, const __grid_constant__ Dp d, uint32_t* out) {
  uint32_t s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 k = __ldcs(reinterpret_cast<const uint2*>(keys) + i);
    if (DEC) {
      const uint32_t w[2] = {k.x, k.y};
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        uint32_t r = 0;
#pragma unroll
        for (int ww = 0; ww < 2; ++ww) {
          uint32_t x = w[ww] & d.mask[m][ww];
#pragma unroll
          for (int st = 0; st < 5; ++st) { const uint32_t t = x & d.mv[m][ww][st]; x = (x ^ t) | (t >> (1u << st)); }
          r |= x << d.shift[m][ww];
        }
        s += r * (m + 1);
      }
    } else {
      s += k.x ^ k.y;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static void compress_moves(uint32_t m, uint32_t mv[5]) {
  uint32_t mk = ~m << 1;
  for (int i = 0; i < 5; ++i) {
    uint32_t mp = mk ^ (mk << 1); mp ^= mp << 2; mp ^= mp << 4; mp ^= mp << 8; mp ^= mp << 16;
    const uint32_t v = mp & m; mv[i] = v; m = (m ^ v) | (v >> (1u << i)); mk = mk & ~mp;
  }
}

template <typename F>
float timeit(F f, int reps) {
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  f(); f(); cudaDeviceSynchronize();
  cudaEventRecord(a);
  for (int i = 0; i < reps; ++i) f();
  cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms, a, b);
  return ms / reps;
}

int main() {
  int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("{\"sms\": %d, \"clock_khz\": %d}\n", sms, clk);
  const int64_t nq = 32ll << 20;          // nonzeros
  const int64_t maxrows = 4ll << 20;      // 4M rows x 128 B = 512 MB
  char* T; uint32_t* idx; float* out; float* sink;
  CK(cudaMalloc(&T, maxrows * 128));
  CK(cudaMalloc(&idx, nq * 2 * 4));
  CK(cudaMalloc(&out, maxrows * 128));
  CK(cudaMalloc(&sink, 152 * 64 * 256 * 4));
  fill_f<<<1024, 256>>>((float*)T, maxrows * 32);
  CK(cudaDeviceSynchronize());
  const uint32_t tsz[4] = {256, 16384, 131072, 4194304};  // rows of 128 B: 32 KB, 2 MB, 16 MB, 512 MB
  for (int ti = 0; ti < 4; ++ti) {
    for (int rb = 0; rb < 2; ++rb) {
      const int ROWB = rb == 0 ? 128 : 64;
      const uint32_t rows = (uint32_t)((int64_t)tsz[ti] * 128 / ROWB);  // same bytes
      fill_idx<<<1024, 256>>>(idx, nq * 2, rows, 12345 + ti);
      CK(cudaDeviceSynchronize());
      for (int bpi = 0; bpi < 4; ++bpi) {
        for (int gm = 0; gm < 2; ++gm) {
          const int grid = sms * (gm == 0 ? 4 : 8);
          float ms = -1; int PB = 0;
          if (ROWB == 128) {
            if (bpi == 0) { PB = 16; ms = timeit([&] { gather2<128, 16><<<grid, 256>>>(T, idx, nq, sink); }, 5); }
            if (bpi == 1) { PB = 32; ms = timeit([&] { gather2<128, 32><<<grid, 256>>>(T, idx, nq, sink); }, 5); }
          } else {
            if (bpi == 0) { PB = 8; ms = timeit([&] { gather2<64, 8><<<grid, 256>>>(T, idx, nq, sink); }, 5); }
            if (bpi == 1) { PB = 16; ms = timeit([&] { gather2<64, 16><<<grid, 256>>>(T, idx, nq, sink); }, 5); }
            if (bpi == 2) { PB = 32; ms = timeit([&] { gather2<64, 32><<<grid, 256>>>(T, idx, nq, sink); }, 5); }
          }
          if (ms < 0) continue;
          CK(cudaGetLastError());
          const double rows_s = 2.0 * nq / (ms * 1e-3);
          printf("{\"probe\": \"gather2\", \"table_bytes\": %lld, \"row_bytes\": %d, \"piece\": %d, \"blocks_per_sm\": %d, "
                 "\"ms\": %.4f, \"Grows_s\": %.2f, \"rows_per_clk_sm\": %.3f, \"TBs\": %.2f}\n",
                 (long long)rows * ROWB, ROWB, PB, grid / sms, ms, rows_s / 1e9, rows_s / (sms * clk * 1e3),
                 rows_s * ROWB / 1e12);
        }
      }
    }
  }
  // RED throughput
  const uint32_t osz[4] = {1024, 32768, 524288, 4194304};
  for (int oi = 0; oi < 4; ++oi) {
    fill_idx<<<1024, 256>>>(idx, nq, osz[oi], 777 + oi);
    CK(cudaMemset(out, 0, (size_t)osz[oi] * 128));
    CK(cudaDeviceSynchronize());
    const float ms = timeit([&] { red_rows<<<sms * 8, 256>>>(out, idx, nq); }, 3);
    CK(cudaGetLastError());
    const double rows_s = nq / (ms * 1e-3);
    printf("{\"probe\": \"red_v4_rows\", \"out_rows\": %u, \"ms\": %.4f, \"Grows_s\": %.2f, \"rows_per_clk_sm\": %.3f}\n",
           osz[oi], ms, rows_s / 1e9, rows_s / (sms * clk * 1e3));
  }
  // decode
  {
    uint64_t* keys = reinterpret_cast<uint64_t*>(idx);  // reuse (nq*8 bytes)
    fill_k<<<1024, 256>>>(keys, nq);
    CK(cudaDeviceSynchronize());
    Dp d{};
    // layout of 4M x 4M x 30k: levels 0..14 (k,i,j) then 15..21 (i,j)
    uint64_t mk[3] = {0, 0, 0};
    int next = 0;
    const int nb[3] = {22, 22, 15};
    const int order[3] = {2, 0, 1};
    for (int l = 0; l < 22; ++l)
      for (int a = 0; a < 3; ++a) { const int m = order[a]; if (l < nb[m]) { mk[m] |= 1ull << next; ++next; } }
    for (int m = 0; m < 3; ++m) {
      uint32_t below = 0;
      for (int w = 0; w < 2; ++w) {
        const uint32_t msk = (uint32_t)(mk[m] >> (32 * w));
        d.mask[m][w] = msk; compress_moves(msk, d.mv[m][w]); d.shift[m][w] = below; below += __builtin_popcount(msk);
      }
    }
    uint32_t* o = reinterpret_cast<uint32_t*>(sink);
    for (int dec = 0; dec < 2; ++dec) {
      const float ms = dec ? timeit([&] { decode3<1><<<sms * 8, 256>>>(keys, nq, d, o); }, 5)
                           : timeit([&] { decode3<0><<<sms * 8, 256>>>(keys, nq, d, o); }, 5);
      CK(cudaGetLastError());
      printf("{\"probe\": \"decode3\", \"decode\": %d, \"ms\": %.4f, \"Gkeys_s\": %.2f, \"keys_per_clk_sm\": %.3f}\n", dec, ms,
             nq / (ms * 1e-3) / 1e9, nq / (ms * 1e-3) / (sms * clk * 1e3));
    }
  }
  CK(cudaDeviceSynchronize());
  printf("{\"done\": true}\n");
  return 0;
}
