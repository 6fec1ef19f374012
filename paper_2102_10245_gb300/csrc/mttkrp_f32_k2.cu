// Instantiation of the MTTKRP kernel family for float factors and 2-word keys.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_f32_k2(const MttkrpLaunch& l, cudaStream_t s) {
  return mttkrp_dispatch_typed<float, 2>(l, s);
}

cudaError_t mttkrp_batch_dispatch_f32_k2(const BatchLaunch& l, cudaStream_t s) {
  return mttkrp_batch_dispatch_typed<float, 2>(l, s);
}

}  // namespace alto
