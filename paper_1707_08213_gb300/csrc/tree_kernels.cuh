// FP32 tree kernels for the 2D sliding window DFT (arXiv 1707.08213, Section 4.2).
//
// Two passes over the two level groups of the tree:
//   row_tree : levels 1..m1 (Eq. rowfswft2d), along dimension 1 of every input row; its
//              level m1 is z[r][q1][k1] = the n1-point DFT of x[r][q1 .. q1+n1-1].
//   col_tree : levels m1+1..m1+m0 (Eq. colfswft2d), along dimension 0 of every channel
//              (q1, k1) of z; its level m0+m1 is the window's 2D DFT, scaled and stored.
// Both walk window positions with SlidingTree (tree_core.cuh), registers only.
//
// z layout: kZPad(n0) = n0/2 padding rows, then rows x P1 x n1 complex64.  The padding lets
// the column pass read its level-0 look-back z[r - n0/2] without a bounds clamp (values
// read there only feed incomplete border trees, which are never stored).
//
// Each column-pass warp covers 32 consecutive channels (q1, k1): its z loads and its
// output stores move 256 contiguous bytes per k0 (full 32-byte sectors).  Outputs go out
// with streaming stores so they do not evict z from L2.
#pragma once

#include <cstdint>

#include "swdft_internal.h"
#include "tree_core.cuh"

namespace swdft {

// w_64^{-j}, j < 64: the twiddles of every power-of-two length (kernel parameter).
struct Omega64 {
    float2 w[kMaxN];
};

struct RowParams {
    RowGeom g;
    Omega64 om;
};

struct ColParams {
    ColGeom g;
    Omega64 om;
};

template <bool CPLX>
__device__ __forceinline__ float2 load_x(const void *row, int64_t i) {
    if constexpr (CPLX) {
        return __ldg(reinterpret_cast<const float2 *>(row) + i);
    } else {
        return make_float2(__ldg(reinterpret_cast<const float *>(row) + i), 0.f);
    }
}

// Row pass, one block tile.  Thread = (row, residue c, chunk of window columns).  Lanes hold
// the residue in the low B bits, then the row, so the 2^B threads of one row store adjacent
// k1 together.  Tile (row_block, chunk_idx) covers rows row_block * (threads >> B) ... of the
// pass and window columns [chunk_idx * chunk, ...).
template <int M, int B, bool CPLX>
__device__ __forceinline__ void row_tile(const RowGeom &p, int row_block, int chunk_idx,
                                         const float2 *om64) {
    using Tree = SlidingTree<M, B>;
    constexpr int n = 1 << M;
    const int c = threadIdx.x & ((1 << B) - 1);
    const int row = row_block * (blockDim.x >> B) + (threadIdx.x >> B);
    if (row >= p.rows) return;
    const int qa = chunk_idx * p.chunk;
    if (qa >= p.P1) return;
    const int qb = min(qa + p.chunk, p.P1);
    const int steps = (qb - qa) + (n - 1);

    const char *xrow = reinterpret_cast<const char *>(p.x) +
                       (p.r_base + row) * p.ld * (int64_t)(CPLX ? sizeof(float2) : sizeof(float));
    float2 *dst = p.z + (int64_t)row * p.zrow + (int64_t)qa * n + c;

    Tree tree;
    tree.init(c, om64);
    for (int jb = 0; jb < steps; jb += Tree::kPeriod) {
        static_for<0, Tree::kPeriod>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = qa + j;  // window end column
                const float2 xp = load_x<CPLX>(xrow, p1);
                const float2 xs = (M >= 1) ? load_x<CPLX>(xrow, max(p1 - Tree::kHalf, 0))
                                           : make_float2(0.f, 0.f);
                float2 o[Tree::kOut];
                tree.template step<J>(xp, xs, o);
                if (j >= n - 1) {
#pragma unroll
                    for (int t = 0; t < Tree::kOut; ++t) dst[t << B] = o[t];
                    dst += n;
                }
            }
        });
    }
}

template <int M, int B, bool CPLX>
__global__ void __launch_bounds__(128) row_tree_kernel(const __grid_constant__ RowParams p) {
    row_tile<M, B, CPLX>(p.g, blockIdx.x, blockIdx.y, p.om.w);
}

// Rows of z staged in shared memory per column-pass block: a ring that holds the level-0
// look-back (n/2 rows) plus two step groups (the group being computed and the one being
// fetched), rounded up to a power of two.
__host__ __device__ constexpr int col_ring_rows(int M) {
    const int need = (M >= 1 ? (1 << (M - 1)) : 0) + 2 * tg_period(M);
    int r = 1;
    while (r < need) r <<= 1;
    return r;
}

__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Column pass, one block tile.  Thread = (channel ch = q1*n1 + k1, residue c, chunk of
// window rows).  Warp w of a block takes residue w mod 2^B (uniform per warp) and channel
// group w / 2^B.  The tile's z rows arrive in a shared-memory ring by cp.async one step group
// ahead of use; all residue warps read the same staged rows.  One __syncthreads per step
// group, no spin-waits; the tile ends with a barrier, so the ring is free for the next tile.
template <int M, int B>
__device__ __forceinline__ void col_tile(const ColGeom &p, int64_t ch_block, int chunk_idx,
                                         const float2 *om64, float2 *ring) {
    using Tree = SlidingTree<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    constexpr int kP = Tree::kPeriod;
    constexpr int kH = Tree::kHalf;
    constexpr int RD = col_ring_rows(M);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int c = warp & (R - 1);
    const int CH = 32 * p.groups;                       // channels of this tile
    const int my = (warp >> B) * 32 + lane;             // this thread's channel in the tile
    const int64_t ch0 = ch_block * CH;
    const int64_t ch = ch0 + my;
    const int qa = chunk_idx * p.chunk;
    if (qa >= p.rows_out) return;                       // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const int steps = (qb - qa) + (n - 1);
    const int zr_end = qb + n - 1;                      // one past the last z row used
    const bool active = ch < p.nch;

    // stage z rows [r_lo, r_hi) of this tile's channels into the ring
    auto fetch = [&](int r_lo, int r_hi) {
        r_hi = min(r_hi, zr_end);
        const int total = (r_hi - r_lo) * CH;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int rr = r_lo + e / CH;
            const int cc = e - (e / CH) * CH;
            const bool ok = ch0 + cc < p.nch;
            const float2 *src = p.z + (int64_t)rr * p.nch + (ok ? ch0 + cc : 0);
            cp_async_8(&ring[(rr & (RD - 1)) * CH + cc], src, ok);
        }
        cp_async_commit();
    };

    const int n1 = 1 << p.m1;
    const int64_t q1 = ch >> p.m1;
    const int64_t k1 = ch & (n1 - 1);
    const int kstride = R * n1;  // elements between outputs t and t+1 (k0 step 2^B)
    float2 *dst = p.out + (int64_t)qa * p.orow + q1 * ((int64_t)n * n1) + (int64_t)c * n1 + k1;
    const float s = p.scale;

    Tree tree;
    tree.init(c, om64);
    fetch(qa - kH, qa + kP);
    cp_async_wait_all();
    __syncthreads();
    for (int jb = 0; jb < steps; jb += kP) {
        if (jb + kP < steps) fetch(qa + jb + kP, qa + jb + 2 * kP);
        static_for<0, kP>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int zr = qa + j;  // z row = window end row, relative to the band
                const float2 xp = ring[(zr & (RD - 1)) * CH + my];
                const float2 xs = (M >= 1) ? ring[((zr - kH) & (RD - 1)) * CH + my] : make_float2(0.f, 0.f);
                float2 o[Tree::kOut];
                tree.template step<J>(xp, xs, o);
                if (j >= n - 1 && active) {
#pragma unroll
                    for (int t = 0; t < Tree::kOut; ++t) __stcs(dst + t * kstride, c_scale(s, o[t]));
                    dst += p.orow;
                }
            }
        });
        cp_async_wait_all();
        __syncthreads();
    }
}

template <int M, int B>
__global__ void __launch_bounds__(256, 2) col_tree_kernel(const __grid_constant__ ColParams p) {
    extern __shared__ float2 ring[];  // col_ring_rows(M) x (32 * groups)
    col_tile<M, B>(p.g, blockIdx.x, blockIdx.y, p.om.w, ring);
}

template <int M, int B>
void row_launch_mb(const RowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
void col_launch_mb(const ColParams &p, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
int col_blocks_per_sm(int threads, int groups);

#define SWDFT_ROW_INSTANTIATE(M_, B_)                                                        \
    template <>                                                                              \
    void row_launch_mb<M_, B_>(const RowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s) { \
        if (cplx)                                                                            \
            row_tree_kernel<M_, B_, true><<<g, b, 0, s>>>(p);                                \
        else                                                                                 \
            row_tree_kernel<M_, B_, false><<<g, b, 0, s>>>(p);                               \
    }

#define SWDFT_COL_INSTANTIATE(M_, B_)                                                     \
    template <>                                                                           \
    void col_launch_mb<M_, B_>(const ColParams &p, dim3 g, dim3 b, cudaStream_t s) {      \
        const size_t smem = sizeof(float2) * col_ring_rows(M_) * 32 * p.g.groups;          \
        col_tree_kernel<M_, B_><<<g, b, smem, s>>>(p);                                    \
    }                                                                                     \
    template <>                                                                           \
    int col_blocks_per_sm<M_, B_>(int threads, int groups) {                              \
        int nb = 0;                                                                       \
        const size_t smem = sizeof(float2) * col_ring_rows(M_) * 32 * groups;             \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, col_tree_kernel<M_, B_>,   \
                                                          threads, smem) != cudaSuccess)  \
            return 0;                                                                     \
        return nb;                                                                        \
    }

// (M, B) pairs with B <= min(M, 3)
#define SWDFT_MB_CASES(F)                                                              \
    F(0, 0) F(1, 0) F(1, 1) F(2, 0) F(2, 1) F(2, 2) F(3, 0) F(3, 1) F(3, 2) F(3, 3)     \
    F(4, 0) F(4, 1) F(4, 2) F(4, 3) F(5, 0) F(5, 1) F(5, 2) F(5, 3) F(6, 0) F(6, 1)     \
    F(6, 2) F(6, 3)

}  // namespace swdft
