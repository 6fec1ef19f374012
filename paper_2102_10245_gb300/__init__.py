"""GB300 (sm_103a) implementation of the ALTO sparse tensor format and of
MTTKRP / CP-ALS over it (Helal et al., ICS '21).

The compute lives in ``libalto.so`` (CUDA kernels behind the C ABI declared
in ``include/alto.h``); this package is its ctypes binding.
"""
from .alto import (AltoError, AltoTensor, Batch, BF16, F32, F64, VAR_ATOMIC, VAR_AUTO, VAR_SMEM,  # noqa: F401
                   VAR_TEMP, VAR_WARPAGG, VARIANT_NAMES, decode_host, launch_count, layout_for_dims,
                   lib, torch_allocator, gram, GRAM_AUTO, GRAM_CUDA_CORES, GRAM_TENSOR_CORES)
