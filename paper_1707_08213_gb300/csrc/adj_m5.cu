// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {5}.
#include "adjoint_kernels.cuh"

namespace swdft {

SWDFT_ADJ_INSTANTIATE(5)

SWDFT_ADJ_RING_INSTANTIATE(5)

}  // namespace swdft
