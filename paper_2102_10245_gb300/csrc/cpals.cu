// CP-ALS driver over ALTO MTTKRP (Sec. 2.2).  Per mode n:
//   M_n = MTTKRP_n                                   (mttkrp kernels)
//   V   = Hadamard product of G_m = U_m^T U_m, m != n (FP64, one block)
//   V = L L^T (Cholesky, FP64), V^{-1} = L^{-T} L^{-1} (FP64)
//   A   = M_n V^{-1}      per row; FP64 for FP64 factors, otherwise the FP64
//                         inverse rounded to FP32 and applied in FP32
//   lambda_r = ||A_:r||_2 (first iteration) or max(1, max_i |A_ir|)
//   U_n = A / lambda (stored in the factor dtype), G_n = U_n^T U_n (FP64 sums
//         of FP32 partials)
// and after the last mode the fit 1 - ||X - model|| / ||X|| from ||X||^2,
// lambda^T (Hadamard of all G) lambda and <X, model> = sum_r lambda_r
// sum_i U_N[i,r] M_N[i,r].
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.h"

namespace alto {

namespace {

constexpr int kT = 256;
constexpr int kMaxR = 64;
constexpr int kGramRows = 64;

template <typename FT>
struct CT {
  using type = float;
};
template <>
struct CT<double> {
  using type = double;
};

template <typename FT>
__device__ __forceinline__ typename CT<FT>::type to_ct(FT v) {
  return static_cast<typename CT<FT>::type>(v);
}
template <>
__device__ __forceinline__ float to_ct<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename FT>
__device__ __forceinline__ FT from_float(float v);
template <>
__device__ __forceinline__ float from_float<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// Accumulate the Gram contribution of one staged tile (rows x R, computing
// type C) into per-thread partials: thread t owns entries t, t+256, ...
template <typename C>
__device__ __forceinline__ void gram_tile(const C (*tile)[kMaxR], int R, C* part) {
  const int RR = R * R;
#pragma unroll
  for (int q = 0; q < kMaxR * kMaxR / kT; ++q) {
    const int e = threadIdx.x + q * kT;
    if (e < RR) {
      const int a = e / R, b = e - a * R;
      C s = C(0);
#pragma unroll 8
      for (int r = 0; r < kGramRows; ++r) s += tile[r][a] * tile[r][b];
      part[q] += s;
    }
  }
}

template <typename C>
__device__ __forceinline__ void gram_flush(const C* part, double* acc, int R) {
  const int RR = R * R;
#pragma unroll
  for (int q = 0; q < kMaxR * kMaxR / kT; ++q)
    if (threadIdx.x + q * kT < RR) acc[q] += static_cast<double>(part[q]);
}

// G += A^T A for A (I x R) of type FT.
template <typename FT>
__global__ void __launch_bounds__(kT) gram_kernel(const FT* __restrict__ A, int64_t I, int R,
                                                  double* __restrict__ G) {
  using C = typename CT<FT>::type;
  __shared__ C tile[kGramRows][kMaxR];
  constexpr int Q = kMaxR * kMaxR / kT;
  C part[Q];
  double acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    part[q] = C(0);
    acc[q] = 0.0;
  }
  int since = 0;
  for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * kGramRows; r0 < I;
       r0 += static_cast<int64_t>(gridDim.x) * kGramRows) {
    const int64_t rows = I - r0 < kGramRows ? I - r0 : kGramRows;
    __syncthreads();
    for (int i = threadIdx.x; i < kGramRows * R; i += kT) {
      const int rr = i / R, cc = i - rr * R;
      tile[rr][cc] = rr < rows ? to_ct<FT>(A[(r0 + rr) * R + cc]) : C(0);
    }
    __syncthreads();
    gram_tile<C>(tile, R, part);
    if (++since == 16) {
      gram_flush<C>(part, acc, R);
#pragma unroll
      for (int q = 0; q < Q; ++q) part[q] = C(0);
      since = 0;
    }
  }
  gram_flush<C>(part, acc, R);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = threadIdx.x + q * kT;
    if (e < R * R) atomicAdd(G + e, acc[q]);
  }
}

// V = Hadamard of G_m (m != skip); Cholesky; V^{-1}.  One block.
__global__ void __launch_bounds__(kT) chol_inv_kernel(const double* __restrict__ G, int N, int skip, int R,
                                                      double* __restrict__ vinv64,
                                                      float* __restrict__ vinv32, int* status) {
  __shared__ double V[kMaxR * kMaxR];
  __shared__ double Li[kMaxR * kMaxR];
  __shared__ int bad;
  const int RR = R * R;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < RR; e += kT) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != skip) v *= G[static_cast<size_t>(m) * RR + e];
    V[e] = v;
  }
  __syncthreads();
  for (int k = 0; k < R; ++k) {
    if (threadIdx.x == 0) {
      const double d = V[k * R + k];
      if (!(d > 0.0)) bad = 1;
      V[k * R + k] = sqrt(d);
    }
    __syncthreads();
    const double dk = V[k * R + k];
    for (int i = k + 1 + threadIdx.x; i < R; i += kT) V[i * R + k] /= dk;
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += kT) {
      const int i = e / R, j = e - i * R;
      if (i > k && j > k && j <= i) V[e] -= V[i * R + k] * V[j * R + k];
    }
    __syncthreads();
  }
  // Li = L^{-1}, column j solved by thread j
  for (int j = threadIdx.x; j < R; j += kT) {
    for (int i = 0; i < R; ++i) {
      if (i < j) {
        Li[i * R + j] = 0.0;
        continue;
      }
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) s -= V[i * R + k] * Li[k * R + j];
      Li[i * R + j] = s / V[i * R + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += kT) {
    const int a = e / R, b = e - a * R;
    double s = 0.0;
    for (int k = a > b ? a : b; k < R; ++k) s += Li[k * R + a] * Li[k * R + b];
    vinv64[e] = s;
    vinv32[e] = static_cast<float>(s);
  }
  if (threadIdx.x == 0 && bad) set_status(status, ALTO_ENOTSPD);
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(__double_as_longlong(v)));
}

// A = Mt V^{-1} row by row; column statistics (sum of squares or max |.|).
template <typename C>
__global__ void __launch_bounds__(kT) solve_kernel(const C* __restrict__ Mt, int64_t I, int R,
                                                   const C* __restrict__ vinv, C* __restrict__ A,
                                                   double* __restrict__ colstat, int use_max) {
  __shared__ C sV[kMaxR * kMaxR];
  __shared__ double red[kT];
  for (int e = threadIdx.x; e < R * R; e += kT) sV[e] = vinv[e];
  __syncthreads();
  const int per = kT / R;  // rows per pass
  const int rr = threadIdx.x / R, col = threadIdx.x - rr * R;
  C stat = C(0);
  if (rr < per) {
    for (int64_t row = static_cast<int64_t>(blockIdx.x) * per + rr; row < I;
         row += static_cast<int64_t>(gridDim.x) * per) {
      const C* m = Mt + row * R;
      C acc = C(0);
      for (int k = 0; k < R; ++k) acc += m[k] * sV[k * R + col];
      A[row * R + col] = acc;
      if (use_max)
        stat = fmax(stat, fabs(acc));
      else
        stat += acc * acc;
    }
  }
  red[threadIdx.x] = (rr < per) ? static_cast<double>(stat) : 0.0;
  __syncthreads();
  if (threadIdx.x < R) {
    double s = 0.0;
    for (int q = 0; q < per; ++q) {
      const double v = red[q * R + threadIdx.x];
      s = use_max ? fmax(s, v) : s + v;
    }
    if (use_max)
      atomic_max_nonneg(colstat + threadIdx.x, s);
    else
      atomicAdd(colstat + threadIdx.x, s);
  }
}

// U = A / lambda (stored as FT), G += U^T U, and optionally
// ip += sum_r lambda_r sum_i U[i,r] Mt[i,r].
template <typename FT>
__global__ void __launch_bounds__(kT) normalize_gram_kernel(const typename CT<FT>::type* __restrict__ A,
                                                            int64_t I, int R,
                                                            const double* __restrict__ colstat,
                                                            int use_max, double* __restrict__ lambda,
                                                            FT* __restrict__ U, double* __restrict__ G,
                                                            const typename CT<FT>::type* __restrict__ Mt,
                                                            double* __restrict__ ip) {
  using C = typename CT<FT>::type;
  __shared__ C tile[kGramRows][kMaxR];
  __shared__ C inv[kMaxR];
  __shared__ double lam[kMaxR];
  __shared__ double ipred[kT];
  constexpr int Q = kMaxR * kMaxR / kT;
  for (int r = threadIdx.x; r < R; r += kT) {
    const double l = use_max ? fmax(colstat[r], 1.0) : sqrt(colstat[r]);
    lam[r] = l;
    inv[r] = static_cast<C>(1.0 / l);
    if (blockIdx.x == 0) lambda[r] = l;
  }
  C part[Q];
  double acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    part[q] = C(0);
    acc[q] = 0.0;
  }
  double ipd = 0.0;
  int since = 0;
  for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * kGramRows; r0 < I;
       r0 += static_cast<int64_t>(gridDim.x) * kGramRows) {
    const int64_t rows = I - r0 < kGramRows ? I - r0 : kGramRows;
    __syncthreads();
    C ipart = C(0);
    for (int i = threadIdx.x; i < kGramRows * R; i += kT) {
      const int rr = i / R, cc = i - rr * R;
      C u = C(0);
      if (rr < rows) {
        const int64_t e = (r0 + rr) * R + cc;
        const FT stored = static_cast<FT>(A[e] * inv[cc]);
        U[e] = stored;
        u = to_ct<FT>(stored);
        if (Mt != nullptr) ipart += u * Mt[e] * static_cast<C>(lam[cc]);
      }
      tile[rr][cc] = u;
    }
    ipd += static_cast<double>(ipart);
    __syncthreads();
    gram_tile<C>(tile, R, part);
    if (++since == 16) {
      gram_flush<C>(part, acc, R);
#pragma unroll
      for (int q = 0; q < Q; ++q) part[q] = C(0);
      since = 0;
    }
  }
  gram_flush<C>(part, acc, R);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = threadIdx.x + q * kT;
    if (e < R * R) atomicAdd(G + e, acc[q]);
  }
  if (Mt != nullptr) {
    ipred[threadIdx.x] = ipd;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) ipred[threadIdx.x] += ipred[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(ip, ipred[0]);
  }
}

// ---------------------------------------------------------------------------
// Warp-per-row versions for R in {8, 16, 32, 64}.  W = min(R, 32) lanes hold
// one row (lane j: columns j + q*W, q < R/W), a warp covers 32/W rows at a
// time, and row values are broadcast with shuffles inside the row's lanes.
template <int R>
struct RowLanes {
  static constexpr int W = R < 32 ? R : 32;
  static constexpr int RPW = 32 / W;   // rows per warp pass
  static constexpr int CPL = R / W;    // columns per lane
  static constexpr int NB = 4;         // independent passes per iteration (loads in flight)
};

__device__ __forceinline__ float shfl_w(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_w(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// A = Mt V^{-1} for R in {8,16,32,64}, with the column statistics.
template <typename C, int R>
__global__ void __launch_bounds__(kT) solve_rows_kernel(const C* __restrict__ Mt, int64_t I,
                                                        const C* __restrict__ vinv, C* __restrict__ A,
                                                        double* __restrict__ colstat, int use_max) {
  using L = RowLanes<R>;
  __shared__ C sV[R * R];
  __shared__ double red[kT / 32][R];
  for (int e = threadIdx.x; e < R * R; e += kT) sV[e] = vinv[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / L::W, j = lane % L::W;
  C stat[L::CPL];
#pragma unroll
  for (int q = 0; q < L::CPL; ++q) stat[q] = C(0);
  const int64_t wid = static_cast<int64_t>(blockIdx.x) * (kT / 32) + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kT / 32);
  constexpr int NB = L::NB;
  for (int64_t r0 = wid * L::RPW * NB; r0 < I; r0 += nw * L::RPW * NB) {
    C m[NB][L::CPL], acc[NB][L::CPL];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int64_t row = r0 + b * L::RPW + grp;
#pragma unroll
      for (int q = 0; q < L::CPL; ++q) {
        m[b][q] = row < I ? Mt[row * R + j + q * L::W] : C(0);
        acc[b][q] = C(0);
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      C v[L::CPL];
#pragma unroll
      for (int q = 0; q < L::CPL; ++q) v[q] = sV[k * R + j + q * L::W];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const C mk = shfl_w(m[b][k / L::W], grp * L::W + (k % L::W));
#pragma unroll
        for (int q = 0; q < L::CPL; ++q) acc[b][q] = fma(mk, v[q], acc[b][q]);
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int64_t row = r0 + b * L::RPW + grp;
      if (row < I) {
#pragma unroll
        for (int q = 0; q < L::CPL; ++q) {
          A[row * R + j + q * L::W] = acc[b][q];
          stat[q] = use_max ? fmax(stat[q], fabs(acc[b][q])) : fma(acc[b][q], acc[b][q], stat[q]);
        }
      }
    }
  }
  // column statistics: combine the row groups of the warp, then the warps
#pragma unroll
  for (int q = 0; q < L::CPL; ++q) {
    double v = static_cast<double>(stat[q]);
    for (int o = L::W; o < 32; o <<= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, v, o);
      v = use_max ? fmax(v, y) : v + y;
    }
    if (grp == 0) red[warp][j + q * L::W] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += kT) {
    double v = 0.0;
    for (int w = 0; w < kT / 32; ++w) v = use_max ? fmax(v, red[w][c]) : v + red[w][c];
    if (use_max)
      atomic_max_nonneg(colstat + c, v);
    else
      atomicAdd(colstat + c, v);
  }
}

// U = A / lambda (stored as FT), G += U^T U, and optionally
// ip += sum_r lambda_r sum_i U[i,r] Mt[i,r].  A warp owns one column block of
// the Gram (columns cb*W + j; R/W blocks), accumulates G[:, its columns] over
// its rows in registers (FP32 partials for FP32/BF16 storage), and the
// partials are summed in FP64 through shared memory, then into G.
template <typename FT, int R>
__global__ void __launch_bounds__(kT) normalize_gram_rows_kernel(
    const typename CT<FT>::type* __restrict__ A, int64_t I, const double* __restrict__ colstat, int use_max,
    double* __restrict__ lambda, FT* __restrict__ U, double* __restrict__ G,
    const typename CT<FT>::type* __restrict__ Mt, double* __restrict__ ip) {
  using C = typename CT<FT>::type;
  using L = RowLanes<R>;
  constexpr int NCB = L::CPL;  // column blocks of the Gram
  __shared__ C inv[R];
  __shared__ double lam[R];
  __shared__ double gred[R * R];
  __shared__ double ipred[kT / 32];
  for (int r = threadIdx.x; r < R; r += kT) {
    const double l = use_max ? fmax(colstat[r], 1.0) : sqrt(colstat[r]);
    lam[r] = l;
    inv[r] = static_cast<C>(1.0 / l);
    if (blockIdx.x == 0) lambda[r] = l;
  }
  for (int e = threadIdx.x; e < R * R; e += kT) gred[e] = 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / L::W, j = lane % L::W;
  const int cb = warp % NCB;
  C g[R];
#pragma unroll
  for (int a = 0; a < R; ++a) g[a] = C(0);
  double ipd = 0.0;
  const int64_t wid = static_cast<int64_t>(blockIdx.x) * (kT / 32 / NCB) + warp / NCB;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kT / 32 / NCB);
  constexpr int NB = L::NB;
  for (int64_t r0 = wid * L::RPW * NB; r0 < I; r0 += nw * L::RPW * NB) {
    C u[NB][L::CPL];
    C own[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int64_t row = r0 + b * L::RPW + grp;
      const bool ok = row < I;
#pragma unroll
      for (int q = 0; q < L::CPL; ++q) {
        const int col = j + q * L::W;
        u[b][q] = C(0);
        if (ok) {
          const FT st = static_cast<FT>(A[row * R + col] * inv[col]);
          u[b][q] = to_ct<FT>(st);
          if (q == cb) {  // the warp of column block q stores it
            U[row * R + col] = st;
            if (Mt != nullptr) ipd += static_cast<double>(u[b][q] * Mt[row * R + col]) * lam[col];
          }
        }
      }
      own[b] = u[b][0];
#pragma unroll
      for (int q = 1; q < L::CPL; ++q)
        if (q == cb) own[b] = u[b][q];
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const C ua = shfl_w(u[b][a / L::W], grp * L::W + (a % L::W));
        g[a] = fma(ua, own[b], g[a]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    double v = static_cast<double>(g[a]);
    for (int o = L::W; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (grp == 0) atomicAdd(&gred[a * R + cb * L::W + j], v);
  }
  for (int o = 16; o > 0; o >>= 1) ipd += __shfl_xor_sync(0xffffffffu, ipd, o);
  if (lane == 0) ipred[warp] = ipd;
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += kT) atomicAdd(G + e, gred[e]);
  if (Mt != nullptr && threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += ipred[w];
    atomicAdd(ip, t);
  }
}

// R <= 32 (one column per lane): the same two passes with the rows a warp
// works on staged in shared memory, so that each lane reads four (FP32) or
// two (FP64) of a row's values with one broadcast 16-byte load instead of one
// shuffle per value.  Capped at 64 registers (4 blocks per SM); the Gram pass
// uses this form for R <= 16 only (at R = 32 its registers spill).
template <typename C>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int N = 4;
  __device__ static float at(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int N = 2;
  __device__ static double at(const double2& v, int i) { return i == 0 ? v.x : v.y; }
};

// A = Mt V^{-1} with the column statistics (R in {8, 16, 32}).
template <typename C, int R>
__global__ void __launch_bounds__(kT, 4) solve_rows_bcast_kernel(const C* __restrict__ Mt, int64_t I,
                                                              const C* __restrict__ vinv, C* __restrict__ A,
                                                              double* __restrict__ colstat, int use_max) {
  using L = RowLanes<R>;
  using V = Vec16<C>;
  static_assert(L::CPL == 1, "one column per lane");
  constexpr int NB = L::NB;
  constexpr int ROWS = NB * L::RPW;  // rows a warp stages per iteration
  __shared__ __align__(16) C sM[kT / 32][ROWS * R];
  __shared__ double red[kT / 32][R];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / L::W, j = lane % L::W;
  C v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = vinv[k * R + j];
  C stat = C(0);
  C* my = sM[warp];
  const int64_t wid = static_cast<int64_t>(blockIdx.x) * (kT / 32) + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kT / 32);
  for (int64_t r0 = wid * ROWS; r0 < I; r0 += nw * ROWS) {
    const int64_t e0 = r0 * R;
    const int64_t e1 = (I < r0 + ROWS ? I : r0 + ROWS) * R;
#pragma unroll
    for (int e = lane; e < ROWS * R; e += 32) my[e] = e0 + e < e1 ? Mt[e0 + e] : C(0);
    __syncwarp();
    C acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = C(0);
#pragma unroll
    for (int k = 0; k < R; k += V::N) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const typename V::T x = *reinterpret_cast<const typename V::T*>(my + (b * L::RPW + grp) * R + k);
#pragma unroll
        for (int i = 0; i < V::N; ++i) acc[b] = fma(V::at(x, i), v[k + i], acc[b]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int64_t row = r0 + b * L::RPW + grp;
      if (row < I) {
        A[row * R + j] = acc[b];
        stat = use_max ? fmax(stat, fabs(acc[b])) : fma(acc[b], acc[b], stat);
      }
    }
  }
  double st = static_cast<double>(stat);
  for (int o = L::W; o < 32; o <<= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, st, o);
    st = use_max ? fmax(st, y) : st + y;
  }
  if (grp == 0) red[warp][j] = st;
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += kT) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t = use_max ? fmax(t, red[w][c]) : t + red[w][c];
    if (use_max)
      atomic_max_nonneg(colstat + c, t);
    else
      atomicAdd(colstat + c, t);
  }
}

// U = A / lambda (stored as FT), G += U^T U, optionally the fit's inner
// product (R in {8, 16, 32}).
template <typename FT, int R>
__global__ void __launch_bounds__(kT, 4) normalize_gram_bcast_kernel(
    const typename CT<FT>::type* __restrict__ A, int64_t I, const double* __restrict__ colstat, int use_max,
    double* __restrict__ lambda, FT* __restrict__ U, double* __restrict__ G,
    const typename CT<FT>::type* __restrict__ Mt, double* __restrict__ ip) {
  using C = typename CT<FT>::type;
  using L = RowLanes<R>;
  using V = Vec16<C>;
  static_assert(L::CPL == 1, "one column per lane");
  constexpr int NB = L::NB;
  constexpr int ROWS = NB * L::RPW;
  __shared__ __align__(16) C sU[kT / 32][ROWS * R];
  __shared__ C inv[R];
  __shared__ double lam[R];
  __shared__ double gred[R * R];
  __shared__ double ipred[kT / 32];
  for (int r = threadIdx.x; r < R; r += kT) {
    const double l = use_max ? fmax(colstat[r], 1.0) : sqrt(colstat[r]);
    lam[r] = l;
    inv[r] = static_cast<C>(1.0 / l);
    if (blockIdx.x == 0) lambda[r] = l;
  }
  for (int e = threadIdx.x; e < R * R; e += kT) gred[e] = 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / L::W, j = lane % L::W;
  const C invj = inv[j];
  const double lamj = lam[j];
  C g[R];
#pragma unroll
  for (int a = 0; a < R; ++a) g[a] = C(0);
  double ipd = 0.0;
  C* my = sU[warp];
  const int64_t wid = static_cast<int64_t>(blockIdx.x) * (kT / 32) + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kT / 32);
  for (int64_t r0 = wid * ROWS; r0 < I; r0 += nw * ROWS) {
    C own[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int64_t row = r0 + b * L::RPW + grp;
      C u = C(0);
      if (row < I) {
        const FT st = static_cast<FT>(A[row * R + j] * invj);
        U[row * R + j] = st;
        u = to_ct<FT>(st);
        if (Mt != nullptr) ipd += static_cast<double>(u * Mt[row * R + j]) * lamj;
      }
      own[b] = u;
      my[(b * L::RPW + grp) * R + j] = u;
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < R; a += V::N) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const typename V::T x = *reinterpret_cast<const typename V::T*>(my + (b * L::RPW + grp) * R + a);
#pragma unroll
        for (int i = 0; i < V::N; ++i) g[a + i] = fma(V::at(x, i), own[b], g[a + i]);
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    double v = static_cast<double>(g[a]);
    for (int o = L::W; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (grp == 0) atomicAdd(&gred[a * R + j], v);
  }
  for (int o = 16; o > 0; o >>= 1) ipd += __shfl_xor_sync(0xffffffffu, ipd, o);
  if (lane == 0) ipred[warp] = ipd;
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += kT) atomicAdd(G + e, gred[e]);
  if (Mt != nullptr && threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += ipred[w];
    atomicAdd(ip, t);
  }
}

// fit = 1 - sqrt(max(0, ||X||^2 + lambda^T (Hadamard G) lambda - 2 ip)) / ||X||
__global__ void __launch_bounds__(kT) fit_kernel(const double* __restrict__ G, int N, int R,
                                                 const double* __restrict__ lambda, double normX2,
                                                 const double* __restrict__ ip, double* __restrict__ fit) {
  __shared__ double red[kT];
  double s = 0.0;
  for (int e = threadIdx.x; e < R * R; e += kT) {
    const int a = e / R, b = e - a * R;
    double v = lambda[a] * lambda[b];
    for (int m = 0; m < N; ++m) v *= G[static_cast<size_t>(m) * R * R + e];
    s += v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double res2 = normX2 + red[0] - 2.0 * ip[0];
    const double res = sqrt(res2 > 0.0 ? res2 : 0.0);
    *fit = 1.0 - res / sqrt(normX2);
  }
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

unsigned rows_grid(int64_t I, int rows_per_block, int per_sm) {
  int64_t g = (I + rows_per_block - 1) / rows_per_block;
  const int64_t cap = static_cast<int64_t>(sm_count()) * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<unsigned>(g);
}

template <typename FT>
cudaError_t launch_gram(const void* A, int64_t I, int R, double* G, cudaStream_t s) {
  if (I <= 0) return cudaSuccess;
  gram_kernel<FT><<<rows_grid(I, kGramRows, 4), kT, 0, s>>>(static_cast<const FT*>(A), I, R, G);
  note_launch();
  return cudaGetLastError();
}

#define CK(expr)                                                                 \
  do {                                                                           \
    const cudaError_t e_ = (expr);                                               \
    if (e_ != cudaSuccess) return fail(ALTO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

template <typename FT>
alto_status cpals_typed(alto_tensor_s* t, int R, int iters, void* const* factors, double* lambda,
                        double* fit, cudaStream_t s) {
  using C = typename CT<FT>::type;
  const int N = t->lay.N;
  CpalsWork& w = t->cp;
  const size_t RR = static_cast<size_t>(R) * R;
  // Gram matrices on the tensor cores for BF16 factors (exact products,
  // FP32 block sums, FP64 across blocks) unless the CUDA cores are asked for
  constexpr bool kBF16 = std::is_same<FT, __nv_bfloat16>::value;
  const bool tc = kBF16 && t->gram_engine != ALTO_GRAM_CUDA_CORES && gram_tc_supported(R);
  // initial Gram matrices
  CK(cudaMemsetAsync(w.gram, 0, sizeof(double) * N * RR, s));
  for (int m = 0; m < N; ++m) {
    if (tc)
      CK(launch_gram_bf16_tc(static_cast<const __nv_bfloat16*>(factors[m]), static_cast<int64_t>(t->lay.dims[m]),
                             R, w.gram + m * RR, t->status, s));
    else
      CK(launch_gram<FT>(factors[m], static_cast<int64_t>(t->lay.dims[m]), R, w.gram + m * RR, s));
  }
  const alto_dtype fd = std::is_same<FT, double>::value ? ALTO_F64
                        : std::is_same<FT, float>::value ? ALTO_F32
                                                          : ALTO_BF16;
  for (int it = 0; it < iters; ++it) {
    for (int n = 0; n < N; ++n) {
      const int64_t In = static_cast<int64_t>(t->lay.dims[n]);
      alto_status st = run_mttkrp(t, n, factors, R, fd, w.mt, ALTO_VAR_AUTO, s);
      if (st != ALTO_OK) return st;
      chol_inv_kernel<<<1, kT, 0, s>>>(w.gram, N, n, R, w.vinv64, w.vinv32, t->status);
      note_launch();
      CK(cudaGetLastError());
      CK(cudaMemsetAsync(w.colstat, 0, sizeof(double) * R, s));
      const int use_max = it > 0 ? 1 : 0;
      const C* vinv = std::is_same<C, double>::value ? reinterpret_cast<const C*>(w.vinv64)
                                                      : reinterpret_cast<const C*>(w.vinv32);
      if (In > 0) {
        const C* mt = static_cast<const C*>(w.mt);
        C* at = static_cast<C*>(w.atmp);
        const unsigned gr = rows_grid(In, 32 * 8, 8);
        switch (R) {
          case 8: solve_rows_bcast_kernel<C, 8><<<gr, kT, 0, s>>>(mt, In, vinv, at, w.colstat, use_max); break;
          case 16: solve_rows_bcast_kernel<C, 16><<<gr, kT, 0, s>>>(mt, In, vinv, at, w.colstat, use_max); break;
          case 32: solve_rows_bcast_kernel<C, 32><<<gr, kT, 0, s>>>(mt, In, vinv, at, w.colstat, use_max); break;
          case 64: solve_rows_kernel<C, 64><<<gr, kT, 0, s>>>(mt, In, vinv, at, w.colstat, use_max); break;
          default:
            solve_kernel<C><<<rows_grid(In, kT / R, 8), kT, 0, s>>>(mt, In, R, vinv, at, w.colstat, use_max);
        }
        note_launch();
        CK(cudaGetLastError());
      }
      CK(cudaMemsetAsync(w.gram + n * RR, 0, sizeof(double) * RR, s));
      const bool last = (n == N - 1);
      if (last) CK(cudaMemsetAsync(w.scal, 0, sizeof(double), s));
      {
        const C* at = static_cast<const C*>(w.atmp);
        FT* un = static_cast<FT*>(factors[n]);
        double* gn = w.gram + n * RR;
        const C* mt = last ? static_cast<const C*>(w.mt) : nullptr;
        const unsigned gr = rows_grid(In, 32 * 8, 8);
        if (tc) {
          CK(launch_normalize_gram_bf16_tc(reinterpret_cast<const float*>(at), In, R, w.colstat, use_max, lambda,
                                           reinterpret_cast<__nv_bfloat16*>(un), gn,
                                           reinterpret_cast<const float*>(mt), w.scal, t->status, s));
          continue;
        }
        switch (R) {
          case 8: normalize_gram_bcast_kernel<FT, 8><<<gr, kT, 0, s>>>(at, In, w.colstat, use_max, lambda, un, gn, mt, w.scal); break;
          case 16: normalize_gram_bcast_kernel<FT, 16><<<gr, kT, 0, s>>>(at, In, w.colstat, use_max, lambda, un, gn, mt, w.scal); break;
          // R = 32: the Gram registers leave no room for the staged rows; the shuffle form stays
          case 32: normalize_gram_rows_kernel<FT, 32><<<gr, kT, 0, s>>>(at, In, w.colstat, use_max, lambda, un, gn, mt, w.scal); break;
          case 64: normalize_gram_rows_kernel<FT, 64><<<gr, kT, 0, s>>>(at, In, w.colstat, use_max, lambda, un, gn, mt, w.scal); break;
          default:
            normalize_gram_kernel<FT><<<rows_grid(In, kGramRows, 4), kT, 0, s>>>(at, In, R, w.colstat, use_max, lambda, un,
                                                                               gn, mt, w.scal);
        }
      }
      note_launch();
      CK(cudaGetLastError());
    }
    fit_kernel<<<1, kT, 0, s>>>(w.gram, N, R, lambda, t->normX2, w.scal, w.fits + it);
    note_launch();
    CK(cudaGetLastError());
  }
  if (fit != nullptr && iters > 0) {
    CK(cudaMemcpyAsync(fit, w.fits, sizeof(double) * iters, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return ALTO_OK;
}

}  // namespace

__device__ int g_gram_status;

alto_status gram_any(const void* U, int64_t I, int R, alto_dtype dtype, int engine, double* G, cudaStream_t s) {
  if (U == nullptr && I > 0) return fail(ALTO_EINVAL, "null factor");
  if (G == nullptr) return fail(ALTO_EINVAL, "null Gram output");
  if (I < 0 || R < 1 || R > kMaxR) return fail(ALTO_EINVAL, "bad shape %lld x %d", static_cast<long long>(I), R);
  if (engine < ALTO_GRAM_AUTO || engine > ALTO_GRAM_TENSOR_CORES) return fail(ALTO_EINVAL, "bad engine %d", engine);
  const bool tc = dtype == ALTO_BF16 && engine != ALTO_GRAM_CUDA_CORES && gram_tc_supported(R);
  if (engine == ALTO_GRAM_TENSOR_CORES && !tc)
    return fail(ALTO_EINVAL, "the tensor-core Gram needs BF16 factors and R in {8, 16, 32, 64}");
  int* status = nullptr;
  CK(cudaGetSymbolAddress(reinterpret_cast<void**>(&status), g_gram_status));
  CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(G, 0, sizeof(double) * R * R, s));
  if (tc) {
    CK(launch_gram_bf16_tc(static_cast<const __nv_bfloat16*>(U), I, R, G, status, s));
  } else {
    switch (dtype) {
      case ALTO_F64: CK(launch_gram<double>(U, I, R, G, s)); break;
      case ALTO_F32: CK(launch_gram<float>(U, I, R, G, s)); break;
      case ALTO_BF16: CK(launch_gram<__nv_bfloat16>(U, I, R, G, s)); break;
      default: return fail(ALTO_EINVAL, "bad dtype");
    }
  }
  int h = 0;
  CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h != 0) return fail(static_cast<alto_status>(h), "device wait ran out in the tensor-core Gram");
  return ALTO_OK;
}

alto_status run_cpals(alto_tensor_s* t, int R, int iters, void* const* factors, alto_dtype fdtype,
                      double* lambda, double* fit, cudaStream_t s) {
  const int N = t->lay.N;
  if (R < 1 || R > kMaxR) return fail(ALTO_EINVAL, "CP-ALS rank %d outside [1, %d]", R, kMaxR);
  if (iters < 0) return fail(ALTO_EINVAL, "iters must be >= 0");
  if (factors == nullptr || lambda == nullptr) return fail(ALTO_EINVAL, "null factors or lambda");
  for (int m = 0; m < N; ++m)
    if (factors[m] == nullptr) return fail(ALTO_EINVAL, "factor %d is null", m);
  if (fdtype == ALTO_F64 && t->vdtype != ALTO_F64)
    return fail(ALTO_EINVAL, "FP64 factors need FP64 values");
  if (fdtype != ALTO_F64 && t->vdtype != ALTO_F32 && t->vdtype != ALTO_BF16)
    return fail(ALTO_EINVAL, "FP32/BF16 factors need FP32 or BF16 values");
  CpalsWork& w = t->cp;
  const size_t osz = fdtype == ALTO_F64 ? 8 : 4;
  uint64_t maxI = 0;
  for (int m = 0; m < N; ++m) maxI = t->lay.dims[m] > maxI ? t->lay.dims[m] : maxI;
  if (w.R != R || w.fdtype != fdtype || w.fits_cap < iters || w.mt == nullptr) {
    dev_free(t, w.mt);
    dev_free(t, w.atmp);
    dev_free(t, w.gram);
    dev_free(t, w.vinv64);
    dev_free(t, w.vinv32);
    dev_free(t, w.colstat);
    dev_free(t, w.scal);
    dev_free(t, w.fits);
    std::memset(&w, 0, sizeof(w));
    const int cap = iters > 16 ? iters : 16;
    w.mt = dev_alloc(t, maxI * R * osz);
    w.atmp = dev_alloc(t, maxI * R * osz);
    w.gram = static_cast<double*>(dev_alloc(t, sizeof(double) * N * R * R));
    w.vinv64 = static_cast<double*>(dev_alloc(t, sizeof(double) * R * R));
    w.vinv32 = static_cast<float*>(dev_alloc(t, sizeof(float) * R * R));
    w.colstat = static_cast<double*>(dev_alloc(t, sizeof(double) * R));
    w.scal = static_cast<double*>(dev_alloc(t, sizeof(double) * 4));
    w.fits = static_cast<double*>(dev_alloc(t, sizeof(double) * cap));
    if (!w.mt || !w.atmp || !w.gram || !w.vinv64 || !w.vinv32 || !w.colstat || !w.scal || !w.fits)
      return fail(ALTO_ENOMEM, "CP-ALS workspace allocation failed");
    w.R = R;
    w.fdtype = fdtype;
    w.fits_cap = cap;
  }
  switch (fdtype) {
    case ALTO_F64: return cpals_typed<double>(t, R, iters, factors, lambda, fit, s);
    case ALTO_F32: return cpals_typed<float>(t, R, iters, factors, lambda, fit, s);
    case ALTO_BF16: return cpals_typed<__nv_bfloat16>(t, R, iters, factors, lambda, fit, s);
  }
  return fail(ALTO_EINVAL, "bad factor dtype");
}

}  // namespace alto
