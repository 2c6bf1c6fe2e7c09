// Fused tree (row levels in the column tile): kernel instantiations (4, 2).
#include "tree_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_FUSED_INSTANTIATE(M_, B_)
F(4, 2)
#undef F

}  // namespace swdft
