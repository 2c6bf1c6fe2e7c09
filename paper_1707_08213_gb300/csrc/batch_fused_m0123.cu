// Persistent fused batch kernels: instantiations (split so they compile in parallel).
#include "batch_fused.cuh"

namespace swdft {

SWDFT_BFU_INSTANTIATE(0)
SWDFT_BFU_INSTANTIATE(1)
SWDFT_BFU_INSTANTIATE(2)
SWDFT_BFU_INSTANTIATE(3)

}  // namespace swdft
