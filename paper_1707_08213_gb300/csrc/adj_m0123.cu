// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {0,1,2,3}.
#include "adjoint_kernels.cuh"

namespace swdft {

SWDFT_ADJ_INSTANTIATE(0)
SWDFT_ADJ_INSTANTIATE(1)
SWDFT_ADJ_INSTANTIATE(2)
SWDFT_ADJ_INSTANTIATE(3)

SWDFT_ADJ_RING_INSTANTIATE(0)
SWDFT_ADJ_RING_INSTANTIATE(1)
SWDFT_ADJ_RING_INSTANTIATE(2)
SWDFT_ADJ_RING_INSTANTIATE(3)

}  // namespace swdft
