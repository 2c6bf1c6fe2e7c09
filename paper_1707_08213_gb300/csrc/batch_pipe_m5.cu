// Pipelined persistent batch kernels: instantiations for log2(n0) in {5} (split so they
// compile in parallel).
#include "batch_pipe.cuh"

namespace swdft {

SWDFT_BPIPE_INSTANTIATE(5)

}  // namespace swdft
