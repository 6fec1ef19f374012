// Instantiation of the MTTKRP kernel family for __nv_bfloat16 factors and 1-word keys.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_bf16_k1(const MttkrpLaunch& l, cudaStream_t s) {
  return mttkrp_dispatch_typed<__nv_bfloat16, 1>(l, s);
}

cudaError_t mttkrp_batch_dispatch_bf16_k1(const BatchLaunch& l, cudaStream_t s) {
  return mttkrp_batch_dispatch_typed<__nv_bfloat16, 1>(l, s);
}

}  // namespace alto
