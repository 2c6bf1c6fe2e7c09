// Column-level pass (Eq. colfswft2d): kernel instantiations for log2(n0) in {6}.
#include "tree_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_COL_INSTANTIATE(M_, B_)
F(6, 2) F(6, 3)
#undef F
SWDFT_COL_TMA_STATUS(6)

}  // namespace swdft
