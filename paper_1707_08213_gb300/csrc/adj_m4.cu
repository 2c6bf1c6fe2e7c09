// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {4}.
#include "adjoint_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_ADJ_INSTANTIATE(M_, B_)
F(4, 0) F(4, 1) F(4, 2) F(4, 3)
#undef F

}  // namespace swdft
