// Column-level pass (Eq. colfswft2d): kernel instantiations for log2(n0) in {0,1,2,3}.
#include "tree_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_COL_INSTANTIATE(M_, B_)
F(0, 0) F(1, 0) F(1, 1) F(2, 0) F(2, 1) F(2, 2) F(3, 0) F(3, 1) F(3, 2) F(3, 3)
#undef F
SWDFT_COL_TMA_STATUS(0)
SWDFT_COL_TMA_STATUS(1)
SWDFT_COL_TMA_STATUS(2)
SWDFT_COL_TMA_STATUS(3)

}  // namespace swdft
