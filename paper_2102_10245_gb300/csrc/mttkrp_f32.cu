// Instantiation of the MTTKRP kernel family for float factors.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_f32(const MttkrpLaunch& l, cudaStream_t s) { return mttkrp_dispatch<float>(l, s); }

}  // namespace alto
