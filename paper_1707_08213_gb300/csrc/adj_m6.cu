// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {6}.
#include "adjoint_kernels.cuh"

namespace swdft {

SWDFT_ADJ_INSTANTIATE(6)

SWDFT_ADJ_RING_INSTANTIATE(6)

}  // namespace swdft
