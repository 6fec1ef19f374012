// MTTKRP over the ALTO format (Sec. 2.2, Alg. 1-2): the fused body of the
// ATOMIC and WARPAGG policies.
//
// Same work split and de-linearization as process_unit (8-segment
// thread-block units, warps interleaving 32-nonzero chunks, one lane
// de-linearizing one nonzero, WARPAGG grouping the chunk by output row), laid
// out so that the warp always has factor-row gathers in flight:
//   * every lane owns 4 consecutive columns (16 bytes of output), so one load
//     per lane and row and one vector atomic per lane cover whole rows;
//   * each warp runs its chunks as a two-stage pipeline: the gathers of chunk
//     c are issued, then chunk c+1 is loaded, de-linearized, grouped and
//     staged into the other half of a double staging buffer while they are in
//     flight, and only then is chunk c summed;
//   * a run of equal output rows is summed in registers as
//     acc = keep * acc + v * prod(rows) (keep = 0 at a run's first position),
//     and the previous run is flushed by a predicated vector atomic at that
//     position, so no branch and no reset instructions sit in the loop;
//   * products use packed FP32x2 arithmetic (exact BF16 x BF16 products
//     through the mixed-precision FMA for BF16 rows), accumulation is FP32
//     (FP64 for FP64 factors).
#pragma once

namespace alto {

template <int R, typename FT>
struct FCols {
  // Every lane owns VB consecutive columns (16 bytes of output: 4 FP32 or 2
  // FP64 accumulators), so one vector atomic per lane and one load per row
  // and lane cover whole rows: a warp instruction touches each row it reads
  // or updates exactly once.
  static constexpr int VB = std::is_same_v<FT, double> ? 2 : 4;
  static constexpr int LPN = R / VB;                              // lanes per nonzero
  static constexpr int CPL = VB;                                  // columns per lane
  static constexpr int BB = VB * static_cast<int>(sizeof(FT));      // bytes of a row per lane
  static constexpr int WORDS = BB / 4;
  static constexpr int G = 32 / LPN;                              // lane groups per warp
  static constexpr int P = 32 / G;                                // positions per group and chunk
  static_assert(R % VB == 0 && LPN >= 1 && LPN <= 32 && 32 % LPN == 0, "rank / element width");
};

// Gathered rows in flight per group before the next chunk is decoded: as
// many positions as fit in the register budget left after the positions'
// values and rows, at least one.
#ifndef ALTO_FUSED_ROW_REGS
#define ALTO_FUSED_ROW_REGS 80
#endif
constexpr int kFusedRowRegs = ALTO_FUSED_ROW_REGS;
template <int N, int R, typename FT>
__host__ __device__ constexpr int fused_depth() {
  constexpr int per = (N > 1 ? N - 1 : 1) * FCols<R, FT>::WORDS;
  constexpr int P = FCols<R, FT>::P;
  constexpr int d = (kFusedRowRegs - 2 * P - (P > 8 ? 16 : 0)) / per;
  return d < 1 ? 1 : (d > P ? P : d);
}

// The lane's piece of one factor row into words (row: the lane's first
// column of the row).
template <typename FC>
__device__ __forceinline__ void ld_row(const char* row, uint32_t* w);

// BYTES of a factor row (read-only for the kernel's lifetime) into words.
template <int BYTES>
__device__ __forceinline__ void ld_piece(const char* p, uint32_t* w) {
  if constexpr (BYTES == 4) {
    w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
  } else if constexpr (BYTES == 8) {
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = a.x;
    w[1] = a.y;
  } else if constexpr (BYTES == 16) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    w[0] = a.x;
    w[1] = a.y;
    w[2] = a.z;
    w[3] = a.w;
  } else {
    static_assert(BYTES % 32 == 0, "pieces above 16 bytes are 32-byte loads");
#pragma unroll
    for (int q = 0; q < BYTES / 32; ++q)
      asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(w[8 * q]), "=r"(w[8 * q + 1]), "=r"(w[8 * q + 2]), "=r"(w[8 * q + 3]), "=r"(w[8 * q + 4]),
            "=r"(w[8 * q + 5]), "=r"(w[8 * q + 6]), "=r"(w[8 * q + 7])
          : "l"(p + 32 * q));
  }
}

template <typename FC>
__device__ __forceinline__ void ld_row(const char* row, uint32_t* w) {
  ld_piece<FC::BB>(row, w);
}

__device__ __forceinline__ float2 f2w(uint32_t a, uint32_t b) {
  return make_float2(__uint_as_float(a), __uint_as_float(b));
}

// acc += v * prod_s rows[s] over the lane's CPL columns.
template <int N, int R, typename FT>
__device__ __forceinline__ void fused_accumulate(const uint32_t (&r)[N - 1][FCols<R, FT>::WORDS],
                                                 typename FTraits<FT>::VT v, typename FTraits<FT>::AT* acc) {
  constexpr int CPL = FCols<R, FT>::CPL;
  if constexpr (std::is_same_v<FT, float>) {
    const float2 v2 = make_float2(v, v);
    if constexpr (CPL == 1) {
      float t = __uint_as_float(r[0][0]);
#pragma unroll
      for (int s = 1; s < N - 1; ++s) t *= __uint_as_float(r[s][0]);
      acc[0] = fmaf(t, v, acc[0]);
    } else {
#pragma unroll
      for (int e = 0; e < CPL; e += 2) {
        float2 t = f2w(r[0][e], r[0][e + 1]);
#pragma unroll
        for (int s = 1; s < N - 1; ++s) t = __fmul2_rn(t, f2w(r[s][e], r[s][e + 1]));
        const float2 x = __ffma2_rn(t, v2, make_float2(acc[e], acc[e + 1]));
        acc[e] = x.x;
        acc[e + 1] = x.y;
      }
    }
  } else if constexpr (std::is_same_v<FT, __nv_bfloat16>) {
    const float2 v2 = make_float2(v, v);
#pragma unroll
    for (int e = 0; e < CPL; e += 2) {
      float2 t;
      if constexpr (N == 2) {
        t = widen_bf16x2(r[0][e / 2]);
      } else {
        t = bf16x2_mul_exact(r[0][e / 2], r[1][e / 2]);
#pragma unroll
        for (int s = 2; s < N - 1; ++s) t = __fmul2_rn(t, widen_bf16x2(r[s][e / 2]));
      }
      const float2 x = __ffma2_rn(t, v2, make_float2(acc[e], acc[e + 1]));
      acc[e] = x.x;
      acc[e + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
      double t = __hiloint2double(static_cast<int>(r[0][2 * e + 1]), static_cast<int>(r[0][2 * e]));
#pragma unroll
      for (int s = 1; s < N - 1; ++s)
        t *= __hiloint2double(static_cast<int>(r[s][2 * e + 1]), static_cast<int>(r[s][2 * e]));
      acc[e] = fma(t, v, acc[e]);
    }
  }
}

// The lane's VB accumulators into an output row (p: the lane's first column
// of the row) with one vector atomic, issued only where `on` holds (a
// predicated instruction, no branch).
template <typename FC>
__device__ __forceinline__ void fused_flush(bool on, float* p, const float* acc) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t"
      "@q red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
      "f"(acc[0]), "f"(acc[1]), "f"(acc[2]), "f"(acc[3]), "r"(static_cast<int>(on)));
}
template <typename FC>
__device__ __forceinline__ void fused_flush(bool on, double* p, const double* acc) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t"
      "@q red.global.add.f64 [%0], %1;\n\t@q red.global.add.f64 [%0+8], %2;\n\t}" ::"l"(p),
      "d"(acc[0]), "d"(acc[1]), "r"(static_cast<int>(on)));
}

// Whether the fused body can run an MTTKRP: a specialised shape whose factor
// and output pointers are aligned to the lane blocks, with an output mode
// shorter than 2^32.
inline bool fused_ok(int N, int R, size_t fsize, const void* const* f, const void* out, size_t osize,
                     uint64_t out_len) {
  if (out_len >= (1ull << 32)) return false;
  if (N < 2 || N > 5 || !(R == 8 || R == 16 || R == 32 || R == 64)) return false;
  const size_t vb = fsize == 8 ? 2 : 4;
  const size_t align = vb * fsize;
  for (int s = 0; s < N - 1; ++s)
    if (reinterpret_cast<uintptr_t>(f[s]) % align != 0) return false;
  return reinterpret_cast<uintptr_t>(out) % (vb * osize) == 0;
}

// Registers of one lane group's positions in a staged chunk: value and
// output row of every position, and the gathered rows of the first D
// positions (issued before the next chunk is decoded).
template <int N, int R, typename FT>
struct GroupWork {
  using VT = typename FTraits<FT>::VT;
  static constexpr int P = FCols<R, FT>::P;
  static constexpr int D = fused_depth<N, R, FT>();
  VT v[P];
  uint32_t row[P];
  uint32_t rw[D][N - 1][FCols<R, FT>::WORDS];
};

// Read a position of the group from its staging slot and issue the gathers
// of its input rows into rw.  A position past the chunk's end (valid false)
// reads the chunk's last valid slot again and gets value 0, so it continues
// that slot's run and adds nothing.
template <int N, int R, typename FT>
__device__ __forceinline__ void fused_issue(const uint4 (*stage)[Stage<N, typename FTraits<FT>::VT>::W4], int slot,
                                            bool valid, const char* const* fb, typename FTraits<FT>::VT& v,
                                            uint32_t& row, uint32_t (&rw)[N - 1][FCols<R, FT>::WORDS]) {
  using FC = FCols<R, FT>;
  using VT = typename FTraits<FT>::VT;
  constexpr size_t RB = static_cast<size_t>(R) * sizeof(FT);
  const Pos<N, VT> t = stage_load<N, VT>(stage[slot]);
  v = valid ? t.v : VT(0);
  row = t.id[N - 1];
#pragma unroll
  for (int s = 0; s < N - 1; ++s) ld_row<FC>(fb[s] + static_cast<size_t>(t.id[s]) * RB, rw[s]);
}

template <int N, int R, typename FT, bool FULL>
__device__ __forceinline__ void fused_prologue(GroupWork<N, R, FT>& w,
                                               const uint4 (*stage)[Stage<N, typename FTraits<FT>::VT>::W4], int p0,
                                               int cnt, const char* const* fb) {
#pragma unroll
  for (int j = 0; j < GroupWork<N, R, FT>::D; ++j) {
    const bool valid = FULL || p0 + j < cnt;
    fused_issue<N, R, FT>(stage, valid ? p0 + j : cnt - 1, valid, fb, w.v[j], w.row[j], w.rw[j]);
  }
}

// acc = keep * acc + v * prod_s rows[s] over the lane's columns (keep is 0
// at the first position of a run, 1 inside it).
template <int N, int R, typename FT>
__device__ __forceinline__ void fused_term(const uint32_t (&r)[N - 1][FCols<R, FT>::WORDS],
                                           typename FTraits<FT>::VT v, typename FTraits<FT>::AT keep,
                                           typename FTraits<FT>::AT* acc) {
  constexpr int CPL = FCols<R, FT>::CPL;
  if constexpr (std::is_same_v<FT, double>) {
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
      double t = __hiloint2double(static_cast<int>(r[0][2 * e + 1]), static_cast<int>(r[0][2 * e]));
#pragma unroll
      for (int s = 1; s < N - 1; ++s)
        t *= __hiloint2double(static_cast<int>(r[s][2 * e + 1]), static_cast<int>(r[s][2 * e]));
      acc[e] = fma(acc[e], keep, t * v);
    }
  } else {
    const float2 v2 = make_float2(v, v), k2 = make_float2(keep, keep);
#pragma unroll
    for (int e = 0; e < CPL; e += 2) {
      float2 t;
      if constexpr (std::is_same_v<FT, float>) {
        t = f2w(r[0][e], r[0][e + 1]);
#pragma unroll
        for (int s = 1; s < N - 1; ++s) t = __fmul2_rn(t, f2w(r[s][e], r[s][e + 1]));
      } else if constexpr (N == 2) {
        t = widen_bf16x2(r[0][e / 2]);
      } else {
        t = bf16x2_mul_exact(r[0][e / 2], r[1][e / 2]);
#pragma unroll
        for (int s = 2; s < N - 1; ++s) t = __fmul2_rn(t, widen_bf16x2(r[s][e / 2]));
      }
      const float2 x = __ffma2_rn(make_float2(acc[e], acc[e + 1]), k2, __fmul2_rn(t, v2));
      acc[e] = x.x;
      acc[e + 1] = x.y;
    }
  }
}

// Output row of a staged row id: the hot-row replica slot when the id
// carries the hot mark (WARPAGG), else the output row.
template <bool AGG, int R, typename AT>
__device__ __forceinline__ AT* fused_dst(uint32_t row, AT* outc, AT* hotc) {
  if constexpr (AGG)
    return ((row & 0x80000000u) ? hotc : outc) + static_cast<size_t>(row & 0x7fffffffu) * R;
  else
    return outc + static_cast<size_t>(row) * R;
}

// Sum the group's positions over runs of equal output rows.  A run's sum is
// flushed (predicated vector atomic) at the first position of the next run,
// and the last run after the loop; positions D .. P-1 are gathered here, D
// positions ahead.
template <int N, int R, typename FT, bool AGG, bool FULL>
__device__ __forceinline__ void fused_compute(GroupWork<N, R, FT>& w,
                                              const uint4 (*stage)[Stage<N, typename FTraits<FT>::VT>::W4], int p0,
                                              int cnt, const char* const* fb, typename FTraits<FT>::AT* outc,
                                              typename FTraits<FT>::AT* hotc) {
  using AT = typename FTraits<FT>::AT;
  using FC = FCols<R, FT>;
  constexpr int P = FC::P, CPL = FC::CPL;
  constexpr int D = GroupWork<N, R, FT>::D;
  AT acc[CPL];
#pragma unroll
  for (int e = 0; e < CPL; ++e) acc[e] = AT(0);
#pragma unroll
  for (int j = 0; j < P; ++j) {
    bool same = false;
    if (j > 0) {
      same = w.row[j] == w.row[j - 1];
      fused_flush<FC>(!same, fused_dst<AGG, R>(w.row[j - 1], outc, hotc), acc);
    }
    fused_term<N, R, FT>(w.rw[j % D], w.v[j], same ? AT(1) : AT(0), acc);
    if (j + D < P) {
      const bool valid = FULL || p0 + j + D < cnt;
      fused_issue<N, R, FT>(stage, valid ? p0 + j + D : cnt - 1, valid, fb, w.v[j + D], w.row[j + D],
                            w.rw[j % D]);
    }
  }
  fused_flush<FC>(FULL || p0 < cnt, fused_dst<AGG, R>(w.row[P - 1], outc, hotc), acc);
}

// Thread-block units u0, u0 + ustride, ... (below uend) of one MTTKRP with the
// fused body; POL is kAtomic or kWarpAgg.  All threads of the block call it
// together.  Each warp walks its chunks (chunks w, w+8, ... of every unit) as
// one two-stage pipeline that runs on across unit boundaries: the gathers of
// chunk c are issued, then chunk c+1 is loaded, de-linearized, grouped by
// output row and staged (into the other half of the warp's double staging
// buffer) while they are in flight, then chunk c is summed and flushed.
template <int N, int W32, int R, typename FT, int POL>
__device__ __forceinline__ void process_units_fused(const MttkrpArgs& a, int64_t u0, int64_t ustride, int64_t uend,
                                                    const BlockState<typename FTraits<FT>::AT>& st,
                                                    uint4 (*s_stage)[kWarps][32][Stage<N, typename FTraits<FT>::VT>::W4]) {
  using AT = typename FTraits<FT>::AT;
  using VT = typename FTraits<FT>::VT;
  using FC = FCols<R, FT>;
  constexpr int P = FC::P, NR = N - 1;
  constexpr bool AGG = POL == kWarpAgg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / FC::LPN, c = lane % FC::LPN;
  const int p0 = g * P;
  const uint32_t lt = lanemask_lt();
  const int H = st.H;
  AT* const outc = static_cast<AT*>(a.out) + c * FC::VB;
  AT* const hotc = st.hdata + c * FC::VB;
  const char* fb[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) fb[s] = static_cast<const char*>(a.f[s]) + c * FC::BB;
  constexpr int64_t kStep = kWarps * 32;

  // a chunk of this warp: unit u, first nonzero base, end of the unit ue
  // (u >= uend marks the end of the walk)
  struct Cur {
    int64_t u, base, ue;
  };
  auto first_in = [&](int64_t u) -> Cur {
    for (; u < uend; u += ustride) {
      const int64_t useg1 = (u + 1) * kUnitSegs < a.L ? (u + 1) * kUnitSegs : a.L;
      const int64_t ub = seg_begin(u * kUnitSegs, a.M, a.L), ue = seg_begin(useg1, a.M, a.L);
      const int64_t base = ub + static_cast<int64_t>(warp) * 32;
      if (base < ue) return Cur{u, base, ue};
    }
    return Cur{uend, 0, 0};
  };
  auto next = [&](Cur x) -> Cur {
    x.base += kStep;
    return x.base < x.ue ? x : first_in(x.u + ustride);
  };

  using VR = typename VRaw<VT>::T;
  // decode, group and stage chunk x (key k, raw value word vr of this lane)
  // into buffer b; returns its nonzero count
  auto front = [&](const Cur& x, const CKey<W32>& k, VR vr, int b) -> int {
    const int cnt = static_cast<int>(x.ue - x.base < 32 ? x.ue - x.base : 32);
    const bool ok = lane < cnt;
    const VT v = value_of<VT>(a, vr, x.base + lane);
    uint32_t id[N];
#pragma unroll
    for (int s = 0; s < N; ++s) id[s] = extract_c<W32>(k, a.dp, s);
    int pos = lane;
    if constexpr (AGG) {
      if (H > 0 && ok && (a.hot_key_bit < 0 || ckey_bit<W32>(k, a.hot_key_bit))) {
        const int slot = hot_lookup(st.hkeys, st.hidx, id[N - 1], a.hot_bits);
        if (slot >= 0) id[N - 1] = 0x80000000u | static_cast<uint32_t>(slot);
      }
      // lanes past the chunk's end share one tag that no row has (the host
      // runs this body only for output modes shorter than 2^32), so they form
      // one group placed after every valid one
      const uint32_t peers = __match_any_sync(0xffffffffu, ok ? id[N - 1] : 0xffffffffu);
      const int leader = __ffs(peers) - 1;
      const uint32_t sz = (lane == leader) ? __popc(peers) : 0u;
      uint32_t inc = sz;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t start = __shfl_sync(0xffffffffu, inc - sz, leader);
      pos = static_cast<int>(start + __popc(peers & lt));
    }
    if (ok) stage_store<N, VT>(s_stage[b][warp][pos], id, v);
    return cnt;
  };
  auto load = [&](const Cur& x, CKey<W32>& k, VR& v) {
    if (x.u < uend && x.base + lane < x.ue) {
      k = load_ckey<W32>(a.keys, x.base + lane);
      v = load_value_raw<VT>(a, x.base + lane);
    }
  };

  Cur cc = first_in(u0);
  if (cc.u >= uend) return;
  Cur c1 = next(cc);
  CKey<W32> kc{}, kn{};
  VR vc{}, vn{};
  load(cc, kc, vc);
  load(c1, kn, vn);
  int buf = 0;
  int cnt = front(cc, kc, vc, buf);
  __syncwarp();
  GroupWork<N, R, FT> w;
  if (cnt == 32)
    fused_prologue<N, R, FT, true>(w, s_stage[buf][warp], p0, cnt, fb);
  else
    fused_prologue<N, R, FT, false>(w, s_stage[buf][warp], p0, cnt, fb);
  while (true) {
    const Cur cn = c1;  // the chunk after cc
    int cnt_n = 0;
    if (cn.u < uend) {  // warp-uniform
      kc = kn;
      vc = vn;
      c1 = next(cn);
      load(c1, kn, vn);
      cnt_n = front(cn, kc, vc, buf ^ 1);
    }
    if (cnt == 32)
      fused_compute<N, R, FT, AGG, true>(w, s_stage[buf][warp], p0, cnt, fb, outc, hotc);
    else
      fused_compute<N, R, FT, AGG, false>(w, s_stage[buf][warp], p0, cnt, fb, outc, hotc);
    __syncwarp();
    if (cn.u >= uend) break;
    if (cnt_n == 32)
      fused_prologue<N, R, FT, true>(w, s_stage[buf ^ 1][warp], p0, cnt_n, fb);
    else
      fused_prologue<N, R, FT, false>(w, s_stage[buf ^ 1][warp], p0, cnt_n, fb);
    cnt = cnt_n;
    buf ^= 1;
  }
}

}  // namespace alto
