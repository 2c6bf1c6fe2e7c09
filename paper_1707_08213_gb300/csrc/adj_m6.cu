// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {6}.
#include "adjoint_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_ADJ_INSTANTIATE(M_, B_)
F(6, 0) F(6, 1) F(6, 2) F(6, 3)
#undef F

}  // namespace swdft
