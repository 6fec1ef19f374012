// Device-memory Temp variant of MTTKRP: Alg. 2 with its local storage and
// pull-based accumulation taken literally.
//
//   accumulate: thread-block unit u (8 consecutive line segments) adds every
//               nonzero's contribution into its own Temp_u, a dense block of
//               (hi_u - lo_u + 1) x R elements over the unit's output-mode
//               interval [lo_u, hi_u] (Temp_l(i - T^s_l, r) in Alg. 2); this
//               is the TEMP policy of the kernel in mttkrp_kernels.cuh;
//   pull:       every output row b sums Temp_u(b - lo_u, :) over the units
//               whose interval contains b (the pull-based reduction of
//               Alg. 2), in unit order.
// The plan (offsets of every Temp_u and, per output row, the list of
// covering units) is built on the host from the segment intervals the first
// time a mode runs with this variant; it is refused when the Temp would
// exceed kTempCapBytes.
#include <vector>

#include "mttkrp_kernels.cuh"

namespace alto {

namespace {

template <typename AT>
__global__ void __launch_bounds__(256) temp_pull_kernel(const AT* __restrict__ temp,
                                                        const uint64_t* __restrict__ toff,
                                                        const uint32_t* __restrict__ ulo,
                                                        const uint64_t* __restrict__ row_ptr,
                                                        const uint32_t* __restrict__ row_units,
                                                        uint64_t I, int R, AT* __restrict__ out) {
  const uint64_t total = I * static_cast<uint64_t>(R);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t e = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const uint64_t b = e / R, r = e - b * R;
    const uint64_t k0 = row_ptr[b], k1 = row_ptr[b + 1];
    if (k1 == k0) continue;
    AT s = AT(0);
    for (uint64_t k = k0; k < k1; ++k) {
      const uint32_t u = row_units[k];
      s += temp[toff[u] + (b - ulo[u]) * R + r];
    }
    out[e] = s;
  }
}

}  // namespace

void free_temp_plan(alto_tensor_s* t, int mode) {
  TempPlan& p = t->tp[mode];
  dev_free(t, p.temp);
  dev_free(t, p.toff);
  dev_free(t, p.ulo);
  dev_free(t, p.row_ptr);
  dev_free(t, p.row_units);
  p = TempPlan();
}

alto_status build_temp_plan(alto_tensor_s* t, int mode, int R, size_t osz, cudaStream_t s) {
  TempPlan& p = t->tp[mode];
  if (p.built && p.R == R && p.osz == osz) return ALTO_OK;
  free_temp_plan(t, mode);
  p.built = true;
  p.R = R;
  p.osz = osz;
  const std::vector<uint32_t>& lo = t->unit_lo[mode];
  const std::vector<uint32_t>& hi = t->unit_hi[mode];
  const size_t U = lo.size();
  std::vector<uint64_t> toff(U + 1, 0);
  uint64_t cover = 0;
  for (size_t u = 0; u < U; ++u) {
    const uint64_t w = hi[u] >= lo[u] ? static_cast<uint64_t>(hi[u]) - lo[u] + 1 : 0;
    toff[u + 1] = toff[u] + w * R;
    cover += w;
  }
  p.temp_elems = toff[U];
  if (p.temp_elems * osz > kTempCapBytes) {
    p.feasible = false;
    return ALTO_OK;
  }
  const uint64_t I = t->lay.dims[mode];
  std::vector<uint64_t> row_ptr(I + 1, 0);
  for (size_t u = 0; u < U; ++u)
    if (hi[u] >= lo[u])
      for (uint64_t b = lo[u]; b <= hi[u]; ++b) row_ptr[b + 1]++;
  for (uint64_t b = 0; b < I; ++b) row_ptr[b + 1] += row_ptr[b];
  std::vector<uint32_t> row_units(cover > 0 ? cover : 1);
  std::vector<uint64_t> cur(row_ptr.begin(), row_ptr.end() - 1);
  for (size_t u = 0; u < U; ++u)
    if (hi[u] >= lo[u])
      for (uint64_t b = lo[u]; b <= hi[u]; ++b) row_units[cur[b]++] = static_cast<uint32_t>(u);
  p.temp = dev_alloc(t, p.temp_elems * osz);
  p.toff = static_cast<uint64_t*>(dev_alloc(t, sizeof(uint64_t) * (U + 1)));
  p.ulo = static_cast<uint32_t*>(dev_alloc(t, sizeof(uint32_t) * (U + 1)));
  p.row_ptr = static_cast<uint64_t*>(dev_alloc(t, sizeof(uint64_t) * (I + 1)));
  p.row_units = static_cast<uint32_t*>(dev_alloc(t, sizeof(uint32_t) * row_units.size()));
  if (!p.temp || !p.toff || !p.ulo || !p.row_ptr || !p.row_units) {
    free_temp_plan(t, mode);
    return fail(ALTO_ENOMEM, "Temp plan allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(p.toff, toff.data(), sizeof(uint64_t) * (U + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && U > 0)
    e = cudaMemcpyAsync(p.ulo, lo.data(), sizeof(uint32_t) * U, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p.row_ptr, row_ptr.data(), sizeof(uint64_t) * (I + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p.row_units, row_units.data(), sizeof(uint32_t) * row_units.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors go out of scope
  if (e != cudaSuccess) {
    free_temp_plan(t, mode);
    return fail(ALTO_ECUDA, "Temp plan upload: %s", cudaGetErrorString(e));
  }
  p.feasible = true;
  return ALTO_OK;
}

cudaError_t launch_temp_variant(alto_tensor_s* t, const MttkrpLaunch& l, alto_dtype fdtype, size_t osz,
                                cudaStream_t s) {
  const int mode = l.args.out_mode;
  const int R = l.args.R;
  if (build_temp_plan(t, mode, R, osz, s) != ALTO_OK) return cudaErrorMemoryAllocation;
  TempPlan& p = t->tp[mode];
  MttkrpLaunch fb = l;
  if (!p.feasible || !mttkrp_specialised(l.N, R)) {
    // Temp too large (or no specialised kernel): warp aggregation instead
    fb.variant = mttkrp_specialised(l.N, R) ? ALTO_VAR_WARPAGG : ALTO_VAR_ATOMIC;
    return mttkrp_dispatch(fb, fdtype, s);
  }
  cudaError_t e = cudaMemsetAsync(p.temp, 0, p.temp_elems * osz, s);
  if (e != cudaSuccess) return e;
  fb.variant = ALTO_VAR_TEMP;
  fb.args.temp = p.temp;
  fb.args.toff = p.toff;
  fb.args.ulo = p.ulo;
  e = mttkrp_dispatch(fb, fdtype, s);
  if (e != cudaSuccess) return e;
  const uint64_t I = t->lay.dims[mode];
  const uint64_t total = I * static_cast<uint64_t>(R);
  uint64_t g = (total + 255) / 256;
  if (g > static_cast<uint64_t>(l.sms) * 16) g = static_cast<uint64_t>(l.sms) * 16;
  if (g < 1) g = 1;
  if (osz == 8)
    temp_pull_kernel<double><<<static_cast<unsigned>(g), 256, 0, s>>>(
        static_cast<const double*>(p.temp), p.toff, p.ulo, p.row_ptr, p.row_units, I, R,
        static_cast<double*>(l.args.out));
  else
    temp_pull_kernel<float><<<static_cast<unsigned>(g), 256, 0, s>>>(
        static_cast<const float*>(p.temp), p.toff, p.ulo, p.row_ptr, p.row_units, I, R,
        static_cast<float*>(l.args.out));
  note_launch();
  return cudaGetLastError();
}

}  // namespace alto
