// Pipelined persistent batch kernels: instantiations for log2(n0) in {0, 1, 2, 3} (split so they
// compile in parallel).
#include "batch_pipe.cuh"

namespace swdft {

SWDFT_BPIPE_INSTANTIATE(0)
SWDFT_BPIPE_INSTANTIATE(1)
SWDFT_BPIPE_INSTANTIATE(2)
SWDFT_BPIPE_INSTANTIATE(3)

}  // namespace swdft
