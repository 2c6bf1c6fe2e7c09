// Persistent fused batch kernels: instantiations (split so they compile in parallel).
#include "batch_fused.cuh"

namespace swdft {

SWDFT_BFU_INSTANTIATE(6)

}  // namespace swdft
