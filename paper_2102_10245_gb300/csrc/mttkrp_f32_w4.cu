// Instantiation of the MTTKRP kernel family for float factors and 128-bit stored
// keys (4 32-bit words); one translation unit per (factor type, key width) so
// that the kernel families compile in parallel.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_f32_w4(const MttkrpLaunch& l, cudaStream_t s) {
  return mttkrp_dispatch_typed<float, 4>(l, s);
}

cudaError_t mttkrp_batch_dispatch_f32_w4(const BatchLaunch& l, cudaStream_t s) {
  return mttkrp_batch_dispatch_typed<float, 4>(l, s);
}

}  // namespace alto
