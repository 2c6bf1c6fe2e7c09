// Row-level pass (Eq. rowfswft2d): kernel instantiations and launcher.
#include <algorithm>

#include "tree_kernels.cuh"

namespace swdft {

SWDFT_MB_CASES(SWDFT_ROW_INSTANTIATE)

cudaError_t launch_row_tree(const RowTreeArgs &a, cudaStream_t s) {
    if (a.rows <= 0 || a.P1 <= 0) return cudaSuccess;
    if (a.m1 < 0 || a.m1 > kMaxLog2 || a.rows > INT32_MAX || a.P1 > INT32_MAX) return cudaErrorInvalidValue;
    RowParams p;
    p.g.x = a.x;
    p.g.ld = a.ld;
    p.g.r_base = a.r_base;
    p.g.zrow = a.P1 << a.m1;
    p.g.rows = (int)a.rows;
    p.g.P1 = (int)a.P1;
    p.g.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.P1, a.P1);
    p.g.z = a.z;
    for (int j = 0; j < kMaxN; ++j) p.om.w[j] = a.om64[j];
    const int B = clamp_split(a.m1, a.B);
    const int threads = 128;
    const int rows_per_block = threads >> B;
    dim3 grid((unsigned)((a.rows + rows_per_block - 1) / rows_per_block),
              (unsigned)((a.P1 + p.g.chunk - 1) / p.g.chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    dim3 block(threads);
    switch (a.m1 * 8 + B) {
#define F(M_, B_)                                         \
    case M_ * 8 + B_:                                     \
        row_launch_mb<M_, B_>(p, a.cplx, grid, block, s); \
        break;
        SWDFT_MB_CASES(F)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
