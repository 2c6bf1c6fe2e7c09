// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {5}.
#include "adjoint_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_ADJ_INSTANTIATE(M_, B_)
F(5, 0) F(5, 1) F(5, 2) F(5, 3)
#undef F

}  // namespace swdft
