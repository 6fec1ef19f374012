// Instantiation of the MTTKRP kernel family for double factors and 96-bit stored
// keys (3 32-bit words); one translation unit per (factor type, key width) so
// that the kernel families compile in parallel.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_f64_w3(const MttkrpLaunch& l, cudaStream_t s) {
  return mttkrp_dispatch_typed<double, 3>(l, s);
}

cudaError_t mttkrp_batch_dispatch_f64_w3(const BatchLaunch& l, cudaStream_t s) {
  return mttkrp_batch_dispatch_typed<double, 3>(l, s);
}

}  // namespace alto
