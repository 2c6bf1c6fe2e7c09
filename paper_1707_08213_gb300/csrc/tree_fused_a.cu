// Fused tree (row levels in the column tile): kernel instantiations (0, 0) (1, 1) (2, 2) (3, 2).
#include "tree_kernels.cuh"

namespace swdft {

#define F(M_, B_) SWDFT_FUSED_INSTANTIATE(M_, B_)
F(0, 0) F(1, 1) F(2, 2) F(3, 2)
#undef F

}  // namespace swdft
