// Ternary and mixed-radix row passes: kernel instantiations for every window shape built.
#include "tree3_kernels.cuh"

namespace swdft {

SWDFT_MIXED_CASES(SWDFT_ROW3_INSTANTIATE)

}  // namespace swdft
