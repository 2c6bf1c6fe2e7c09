// Persistent fused groups of a batch: one kernel per (m0, m1) whose blocks take the column
// tiles of every array in the group round-robin and evaluate each tile's z rows from the
// input (ZStageRowDft) instead of reading them, as the per-array fused kernel does.
#pragma once

#include "tree_kernels.cuh"

namespace swdft {

__host__ __device__ constexpr int bfu_B(int m0) { return m0 >= 6 ? 3 : (m0 < 2 ? m0 : 2); }
__host__ __device__ constexpr int bfu_threads(int m0) { return m0 >= 6 ? 256 : 128; }
// Resident blocks the batch kernels are compiled for.  A batch block reads its tile's geometry
// from the descriptor table, so without a bound the compiler keeps it in up to ~20 more
// registers than the per-array kernels (whose geometry is a kernel parameter) and fewer
// blocks fit an SM; these bounds are the largest that compile without spills (n0 = 32: 96
// registers, 5 blocks; n0 = 16: 64-80; n0 <= 8: 64).
__host__ __device__ constexpr int bcol_min_blocks(int m0) { return m0 >= 6 ? 2 : (m0 == 5 ? 5 : 8); }
__host__ __device__ constexpr int bfu_min_blocks(int m0, int m1) {
    return m0 >= 6 ? 2 : (m0 == 5 ? 5 : (m0 == 4 ? (m1 >= 5 ? 6 : 7) : 8));
}

__device__ __forceinline__ int bfu_find_entry(const BatchClassEntry *__restrict__ ent, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&ent[mid].item0) <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int M0, int M1, bool CPLX>
__device__ __forceinline__ void bfu_tile(const BatchImage &d, int64_t cb, int ck, const float2 *om, float2 *ring) {
    ZStageRowDft<M1, CPLX> st;
    st.x = reinterpret_cast<const char *>(d.row.x) +
           d.row.r_base * d.row.ld * (int64_t)(CPLX ? sizeof(float2) : sizeof(float));
    st.ld = d.row.ld;
    st.zrows = d.row.rows;
    st.P1 = d.row.P1;
    st.init(om);
    col_tile_impl<M0, bfu_B(M0)>(d.col, cb, ck, om, ring, st);
}

template <int M0, int M1>
__global__ void __launch_bounds__(bfu_threads(M0), bfu_min_blocks(M0, M1))
    batch_fused_kernel(const BatchImage *__restrict__ imgs, const BatchClassEntry *__restrict__ ent, int nent,
                       int64_t nitems, const __grid_constant__ Omega64 om) {
    extern __shared__ float2 ring[];
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int e = bfu_find_entry(ent, nent, it);
        const BatchImage &d = imgs[__ldg(&ent[e].img)];
        const int64_t local = it - __ldg(&ent[e].item0);
        const int64_t cb = local % d.col_blocks;
        const int ck = (int)(local / d.col_blocks);
        if (d.cplx)
            bfu_tile<M0, M1, true>(d, cb, ck, om.w, ring);
        else
            bfu_tile<M0, M1, false>(d, cb, ck, om.w, ring);
    }
}

// groups of 32 channels per column tile, as batch_col_groups
__host__ __device__ constexpr int bfu_groups(int m0) { return m0 >= 6 ? 1 : (4 >> bfu_B(m0)); }
inline size_t bfu_smem(int m0) { return sizeof(float2) * col_ring_rows(m0) * 32 * bfu_groups(m0); }

// launcher and occupancy for one M0 (all m1), defined in batch_fused_m*.cu
template <int M0>
cudaError_t bfu_launch(int m1, const BatchImage *d_images, const BatchClassEntry *ent, int nent, int64_t nitems,
                       const Omega64 &om, unsigned grid, cudaStream_t s);
template <int M0>
cudaError_t bfu_bps(int m1, int *bps);

#define SWDFT_BFU_INSTANTIATE(M0_)                                                                          \
    template <>                                                                                             \
    cudaError_t bfu_launch<M0_>(int m1, const BatchImage *d_images, const BatchClassEntry *ent, int nent,   \
                                int64_t nitems, const Omega64 &om, unsigned grid, cudaStream_t s) {         \
        const size_t smem = bfu_smem(M0_);                                                                  \
        switch (m1) {                                                                                       \
            case 0: batch_fused_kernel<M0_, 0><<<grid, bfu_threads(M0_), smem, s>>>(d_images, ent, nent, nitems, om); break; \
            case 1: batch_fused_kernel<M0_, 1><<<grid, bfu_threads(M0_), smem, s>>>(d_images, ent, nent, nitems, om); break; \
            case 2: batch_fused_kernel<M0_, 2><<<grid, bfu_threads(M0_), smem, s>>>(d_images, ent, nent, nitems, om); break; \
            case 3: batch_fused_kernel<M0_, 3><<<grid, bfu_threads(M0_), smem, s>>>(d_images, ent, nent, nitems, om); break; \
            case 4: batch_fused_kernel<M0_, 4><<<grid, bfu_threads(M0_), smem, s>>>(d_images, ent, nent, nitems, om); break; \
            case 5: batch_fused_kernel<M0_, 5><<<grid, bfu_threads(M0_), smem, s>>>(d_images, ent, nent, nitems, om); break; \
            default: return cudaErrorInvalidValue;                                                          \
        }                                                                                                   \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    template <>                                                                                             \
    cudaError_t bfu_bps<M0_>(int m1, int *bps) {                                                            \
        const size_t smem = bfu_smem(M0_);                                                                  \
        switch (m1) {                                                                                       \
            case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_fused_kernel<M0_, 0>, bfu_threads(M0_), smem); \
            case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_fused_kernel<M0_, 1>, bfu_threads(M0_), smem); \
            case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_fused_kernel<M0_, 2>, bfu_threads(M0_), smem); \
            case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_fused_kernel<M0_, 3>, bfu_threads(M0_), smem); \
            case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_fused_kernel<M0_, 4>, bfu_threads(M0_), smem); \
            case 5: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_fused_kernel<M0_, 5>, bfu_threads(M0_), smem); \
            default: return cudaErrorInvalidValue;                                                          \
        }                                                                                                   \
    }

}  // namespace swdft
