// Adjoint passes (transposed tree): kernel instantiations for log2(n) in {0,1,2,3}.
#include "adjoint_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_ADJ_INSTANTIATE(M_, B_)
F(0, 0) F(1, 0) F(1, 1) F(2, 0) F(2, 1) F(2, 2) F(3, 0) F(3, 1) F(3, 2) F(3, 3)
#undef F

}  // namespace swdft
