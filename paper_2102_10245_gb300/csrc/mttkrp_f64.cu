// Instantiation of the MTTKRP kernel family for double factors.
#include "mttkrp_kernels.cuh"

namespace alto {

cudaError_t mttkrp_dispatch_f64(const MttkrpLaunch& l, cudaStream_t s) { return mttkrp_dispatch<double>(l, s); }

}  // namespace alto
