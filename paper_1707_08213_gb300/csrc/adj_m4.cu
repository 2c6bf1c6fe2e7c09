// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {4}.
#include "adjoint_kernels.cuh"

namespace swdft {

SWDFT_ADJ_INSTANTIATE(4)

SWDFT_ADJ_RING_INSTANTIATE(4)

}  // namespace swdft
