// Instantiation of the MTTKRP kernel family for __nv_bfloat16 factors.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_bf16(const MttkrpLaunch& l, cudaStream_t s) { return mttkrp_dispatch<__nv_bfloat16>(l, s); }

}  // namespace alto
