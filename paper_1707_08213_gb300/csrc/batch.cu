// Persistent launches over a batch of arrays of uneven sizes and window shapes.
//
// The forward tree of every array is cut into block-sized tiles: row tiles (blocks of input
// rows x chunks of window columns, Eq. rowfswft2d) and column tiles (channel groups x chunks
// of window rows, Eq. colfswft2d).  Arrays are grouped by window exponent (m1 for row tiles,
// m0 for column tiles); each group gets one persistent kernel, compiled for that exponent so
// it has its own register budget, whose grid of (SMs x resident blocks) blocks takes the
// group's tiles round-robin across all its arrays -- small arrays do not leave the GPU idle
// and large ones do not leave a partial last wave per array.  The host runs the groups'
// kernels concurrently on forked streams: first every row group, then (after a join) every
// column group.  A block finds its tile's array by binary search over the group's tile
// offsets and calls the same tile functions the per-array kernels use.  Every array has its
// own z region of the workspace.  No inter-block waits.  Arrays the plan marks fused skip
// both groups: a fused group per (m0, m1) (batch_fused.cuh) runs their column tiles with
// the row levels evaluated in the tile, concurrently with the row groups.
#include <algorithm>

#include "batch_fused.cuh"
#include "tree_kernels.cuh"

namespace swdft {

// Launch choices the batch kernels use for a window side of 2^m (as the per-array defaults):
// column tiles of 128 threads (256 for 64-point trees; bfu_B / bfu_threads / bfu_groups of
// batch_fused.cuh, shared with the fused groups), row tiles of 128 threads.
__host__ __device__ constexpr int brow_B(int m1) { return m1 >= 6 ? 2 : (m1 < 3 ? m1 : 3); }
static constexpr int kRowThreads = 128;
static_assert(32 * (1 << bfu_B(6)) * bfu_groups(6) == bfu_threads(6) &&
                  32 * (1 << bfu_B(5)) * bfu_groups(5) == bfu_threads(5),
              "column tiles: 2^B residue warps x 32-channel groups fill the block");

int batch_row_B(int m1) { return brow_B(m1); }
int batch_col_B(int m0) { return bfu_B(m0); }
int batch_col_groups(int m0) { return bfu_groups(m0); }

template <int M1>
__global__ void __launch_bounds__(kRowThreads)
    batch_row_kernel(const BatchImage *__restrict__ imgs, const BatchClassEntry *__restrict__ ent, int nent,
                     int64_t nitems, const __grid_constant__ Omega64 om) {
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int e = bfu_find_entry(ent, nent, it);
        const BatchImage &d = imgs[__ldg(&ent[e].img)];
        const int64_t local = it - __ldg(&ent[e].item0);
        const int rb = (int)(local % d.row_blocks);
        const int ck = (int)(local / d.row_blocks);
        const RowGeom g = d.row;
        if (d.cplx)
            row_tile<M1, brow_B(M1), true>(g, rb, ck, om.w);
        else
            row_tile<M1, brow_B(M1), false>(g, rb, ck, om.w);
    }
}

template <int M0>
__global__ void __launch_bounds__(bfu_threads(M0), M0 >= 6 ? 2 : 4)
    batch_col_kernel(const BatchImage *__restrict__ imgs, const BatchClassEntry *__restrict__ ent, int nent,
                     int64_t nitems, const __grid_constant__ Omega64 om) {
    extern __shared__ float2 ring[];
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int e = bfu_find_entry(ent, nent, it);
        const BatchImage &d = imgs[__ldg(&ent[e].img)];
        const int64_t local = it - __ldg(&ent[e].item0);
        const int64_t cb = local % d.col_blocks;
        const int ck = (int)(local / d.col_blocks);
        const ColGeom g = d.col;
        col_tile<M0, bfu_B(M0)>(g, cb, ck, om.w, ring);
    }
}

cudaError_t batch_blocks_per_sm(int m, int *row_bps, int *col_bps) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (m) {
#define F(M_)                                                                                              \
    case M_:                                                                                               \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(row_bps, batch_row_kernel<M_>, kRowThreads, 0);  \
        if (e != cudaSuccess) return e;                                                                    \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(col_bps, batch_col_kernel<M_>,                \
                                                             bfu_threads(M_), bfu_smem(M_));
        F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
        default:
            return e;
    }
}

cudaError_t launch_batch_class(bool col, int m, const BatchImage *d_images, const BatchClassEntry *ent, int nent,
                               int64_t nitems, const float2 *om64, int64_t slots, cudaStream_t s) {
    if (nent <= 0 || nitems <= 0) return cudaSuccess;
    Omega64 om;
    for (int j = 0; j < kMaxN; ++j) om.w[j] = om64[j];
    const unsigned grid = (unsigned)std::min<int64_t>(nitems, std::max<int64_t>(1, slots));
    switch (m) {
#define F(M_)                                                                                                 \
    case M_:                                                                                                  \
        if (col)                                                                                              \
            batch_col_kernel<M_><<<grid, bfu_threads(M_), bfu_smem(M_), s>>>(d_images, ent, nent, nitems, om); \
        else                                                                                                  \
            batch_row_kernel<M_><<<grid, kRowThreads, 0, s>>>(d_images, ent, nent, nitems, om);               \
        break;
        F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t batch_fused_blocks_per_sm(int m0, int m1, int *bps) {
    if (m1 < 0 || m1 >= kBatchFusedM1) return cudaErrorInvalidValue;
    switch (m0) {
        case 0: return bfu_bps<0>(m1, bps);
        case 1: return bfu_bps<1>(m1, bps);
        case 2: return bfu_bps<2>(m1, bps);
        case 3: return bfu_bps<3>(m1, bps);
        case 4: return bfu_bps<4>(m1, bps);
        case 5: return bfu_bps<5>(m1, bps);
        case 6: return bfu_bps<6>(m1, bps);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_fused_class(int m0, int m1, const BatchImage *d_images, const BatchClassEntry *ent,
                                     int nent, int64_t nitems, const float2 *om64, int64_t slots, cudaStream_t s) {
    if (nent <= 0 || nitems <= 0) return cudaSuccess;
    Omega64 om;
    for (int j = 0; j < kMaxN; ++j) om.w[j] = om64[j];
    const unsigned grid = (unsigned)std::min<int64_t>(nitems, std::max<int64_t>(1, slots));
    switch (m0) {
        case 0: return bfu_launch<0>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 1: return bfu_launch<1>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 2: return bfu_launch<2>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 3: return bfu_launch<3>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 4: return bfu_launch<4>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 5: return bfu_launch<5>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 6: return bfu_launch<6>(m1, d_images, ent, nent, nitems, om, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swdft
