// Ternary and mixed-radix column passes: kernel instantiations for every window shape built.
#include "tree3_kernels.cuh"

namespace swdft {

SWDFT_MIXED_CASES(SWDFT_COL3_INSTANTIATE)

}  // namespace swdft
