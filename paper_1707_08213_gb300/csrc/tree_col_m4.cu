// Column-level pass (Eq. colfswft2d): kernel instantiations for log2(n0) in {4}.
#include "tree_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_COL_INSTANTIATE(M_, B_)
F(4, 0) F(4, 1) F(4, 2) F(4, 3)
#undef F
SWDFT_COL_TMA_STATUS(4)

}  // namespace swdft
