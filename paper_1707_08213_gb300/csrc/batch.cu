// Persistent launch over a batch of arrays of uneven sizes and window shapes.
//
// The forward tree of every array is cut into block-sized tiles: row tiles (blocks of input
// rows x chunks of window columns, Eq. rowfswft2d) and column tiles (32-channel groups x
// chunks of window rows, Eq. colfswft2d).  Two persistent kernels, launched back to back on
// one stream, each run a grid of (SMs x resident blocks) blocks that take tiles round-robin
// across ALL arrays, so small arrays do not leave the GPU idle and large ones do not leave a
// partial last wave per array.  The block finds its tile's array by binary search over the
// per-array tile offsets and dispatches on the array's window exponent to the same tile
// functions the per-array kernels use.  Every array has its own z region of the workspace.
// No inter-block waits: the stream order separates the two passes.
#include <algorithm>

#include "tree_kernels.cuh"

namespace swdft {

constexpr int kBatchThreads = 256;

int batch_row_B(int m1) { return m1 >= 6 ? 3 : std::min(m1, 2); }
int batch_col_B(int m0) { return m0 >= 6 ? 3 : std::min(m0, 2); }
int batch_col_groups(int m0) { return (kBatchThreads / 32) >> batch_col_B(m0); }

__device__ __forceinline__ int find_image(const BatchImage *__restrict__ imgs, int nimg,
                                          int64_t item, bool col) {
    int lo = 0, hi = nimg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t first = col ? __ldg(&imgs[mid].col_item0) : __ldg(&imgs[mid].row_item0);
        if (first <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <bool CPLX>
__device__ __forceinline__ void row_dispatch(int m1, const RowGeom &g, int rb, int ck, const float2 *om) {
    switch (m1) {
        case 0: row_tile<0, 0, CPLX>(g, rb, ck, om); break;
        case 1: row_tile<1, 1, CPLX>(g, rb, ck, om); break;
        case 2: row_tile<2, 2, CPLX>(g, rb, ck, om); break;
        case 3: row_tile<3, 2, CPLX>(g, rb, ck, om); break;
        case 4: row_tile<4, 2, CPLX>(g, rb, ck, om); break;
        case 5: row_tile<5, 2, CPLX>(g, rb, ck, om); break;
        case 6: row_tile<6, 3, CPLX>(g, rb, ck, om); break;
        default: break;
    }
}

__global__ void __launch_bounds__(kBatchThreads, 2)
    batch_row_kernel(const BatchImage *__restrict__ imgs, int nimg, int64_t nitems,
                     const __grid_constant__ Omega64 om) {
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int i = find_image(imgs, nimg, it, false);
        const BatchImage &d = imgs[i];
        const int64_t local = it - d.row_item0;
        const int rb = (int)(local % d.row_blocks);
        const int ck = (int)(local / d.row_blocks);
        const RowGeom g = d.row;
        if (d.cplx)
            row_dispatch<true>(d.m1, g, rb, ck, om.w);
        else
            row_dispatch<false>(d.m1, g, rb, ck, om.w);
    }
}

__global__ void __launch_bounds__(kBatchThreads, 2)
    batch_col_kernel(const BatchImage *__restrict__ imgs, int nimg, int64_t nitems,
                     const __grid_constant__ Omega64 om) {
    extern __shared__ float2 ring[];
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int i = find_image(imgs, nimg, it, true);
        const BatchImage &d = imgs[i];
        const int64_t local = it - d.col_item0;
        const int64_t cb = local % d.col_blocks;
        const int ck = (int)(local / d.col_blocks);
        const ColGeom g = d.col;
        switch (d.m0) {
            case 0: col_tile<0, 0>(g, cb, ck, om.w, ring); break;
            case 1: col_tile<1, 1>(g, cb, ck, om.w, ring); break;
            case 2: col_tile<2, 2>(g, cb, ck, om.w, ring); break;
            case 3: col_tile<3, 2>(g, cb, ck, om.w, ring); break;
            case 4: col_tile<4, 2>(g, cb, ck, om.w, ring); break;
            case 5: col_tile<5, 2>(g, cb, ck, om.w, ring); break;
            case 6: col_tile<6, 3>(g, cb, ck, om.w, ring); break;
            default: break;
        }
    }
}

static size_t batch_col_smem() {
    size_t m = 0;
    for (int m0 = 0; m0 <= kMaxLog2; ++m0)
        m = std::max(m, sizeof(float2) * col_ring_rows(m0) * 32 * batch_col_groups(m0));
    return m;
}

cudaError_t batch_blocks_per_sm(int *row_bps, int *col_bps) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(row_bps, batch_row_kernel, kBatchThreads, 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(col_bps, batch_col_kernel, kBatchThreads,
                                                         batch_col_smem());
}

cudaError_t launch_batch_tree(const BatchImage *d_images, int nimg, int64_t row_items,
                              int64_t col_items, const float2 *om64, int64_t row_slots,
                              int64_t col_slots, cudaStream_t s) {
    if (nimg <= 0) return cudaSuccess;
    Omega64 om;
    for (int j = 0; j < kMaxN; ++j) om.w[j] = om64[j];
    const size_t smem = batch_col_smem();
    cudaError_t e;
    const int64_t row_grid = std::min<int64_t>(row_items, std::max<int64_t>(1, row_slots));
    const int64_t col_grid = std::min<int64_t>(col_items, std::max<int64_t>(1, col_slots));
    if (row_grid > 0) batch_row_kernel<<<(unsigned)row_grid, kBatchThreads, 0, s>>>(d_images, nimg, row_items, om);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (col_grid > 0) batch_col_kernel<<<(unsigned)col_grid, kBatchThreads, smem, s>>>(d_images, nimg, col_items, om);
    return cudaGetLastError();
}

}  // namespace swdft
