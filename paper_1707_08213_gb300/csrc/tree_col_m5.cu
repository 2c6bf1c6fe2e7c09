// Column-level pass (Eq. colfswft2d): kernel instantiations for log2(n0) in {5}.
#include "tree_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_COL_INSTANTIATE(M_, B_)
F(5, 0) F(5, 1) F(5, 2) F(5, 3)
#undef F
SWDFT_COL_TMA_STATUS(5)

}  // namespace swdft
