// Adjoint (A^H) kernels of the 2D sliding window DFT: the transposed tree of Section 4.2,
// i.e. the overlap-add of every window's inverse DFT of the upstream gradient G.
//
// The forward map is A = C R (row levels R: x -> z, then column levels C: z -> a, each a
// sliding transform along one axis), so A^H = R^H C^H, again two passes:
//   adj_col : per channel (q1, k1), walk z rows downwards with SlidingTreeAdjoint along
//             dimension 0:  gz[r][q1][k1] = c * sum_j0 sum_k0 G[r-j0][q1][k0][k1] w_{n0}^{+j0 k0}
//   adj_row : per z row, walk columns downwards along dimension 1:
//             gx[r][p1] = sum_j1 sum_k1 gz[r][p1-j1][k1] w_{n1}^{+j1 k1}   (real part for real x)
// gz uses the same workspace as the forward pass's z (rows x P1 x n1 complex64).
//
// Lanes hold (residue c in the low B bits, channel or row above): the 2^B partials of one
// output are reduced with shuffles and lane c = 0 stores.  G is read once, coalesced: for a
// fixed node t the lanes of one residue read consecutive k1 of one k0 row.
#pragma once

#include <cstdint>

#include "swdft_internal.h"
#include "adjoint_core.cuh"

namespace swdft {

struct AdjColParams {
    const float2 *G;   // rows_out x P1 x n0 x n1
    float2 *gz;        // (rows_out + n0 - 1) x P1 x n1
    int64_t nch;       // P1 * n1
    int rows_out;      // window rows of G
    int zrows;         // rows_out + n0 - 1
    int chunk;         // gz rows per thread (plus n0 - 1 warm-up steps)
    int m1;
    float scale;
    float2 om64[kMaxN];  // w_64^{-j}: every power-of-two length's twiddles
};

struct AdjRowParams {
    const float2 *gz;  // zrows x P1 x n1
    void *gx;          // zrows rows of N1 elements (row stride ld_out)
    int64_t ld_out;
    int zrows;
    int N1, P1;
    int chunk;         // output columns per thread (plus n1 - 1 warm-up steps)
    float2 om64[kMaxN];  // w_64^{-j}: every power-of-two length's twiddles
};

template <int R>
__device__ __forceinline__ float2 reduce_residues(float2 v) {
#pragma unroll
    for (int off = 1; off < R; off <<= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    return v;
}

template <int M, int B>
__global__ void __launch_bounds__(128) adj_col_kernel(const __grid_constant__ AdjColParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    const int c = threadIdx.x & (R - 1);
    const int64_t ch = (int64_t)blockIdx.x * (blockDim.x >> B) + (threadIdx.x >> B);
    const bool active = ch < p.nch;
    const int ra = blockIdx.y * p.chunk;
    if (ra >= p.zrows) return;  // uniform per block
    const int rb = min(ra + p.chunk, p.zrows);
    const int p_hi = min(rb + n - 2, p.zrows - 1);
    const int steps = p_hi - ra + 1;

    const int n1 = 1 << p.m1;
    const int64_t chc = active ? ch : 0;
    const int64_t q1 = chc >> p.m1;
    const int64_t k1 = chc & (n1 - 1);
    const int64_t win = (int64_t)n * n1;
    const int64_t grow = p.nch * n;  // elements per window row of G
    const float2 *gbase = p.G + q1 * win + (int64_t)c * n1 + k1;
    const int kstride = R * n1;
    const float s = p.scale;

    // G for step j: the window ending at z row p_hi - j (zeros where none ends there)
    auto load_g = [&](int j, float2 (&u)[Tree::kIn]) {
        const int q0 = p_hi - j - (n - 1);
        if (active && j < steps && q0 >= 0 && q0 < p.rows_out) {
            const float2 *g = gbase + (int64_t)q0 * grow;
#pragma unroll
            for (int t = 0; t < Tree::kIn; ++t) u[t] = __ldcs(g + t * kstride);
        } else {
#pragma unroll
            for (int t = 0; t < Tree::kIn; ++t) u[t] = make_float2(0.f, 0.f);
        }
    };

    Tree tree;
    tree.init(c, p.om64);
    // software pipeline: the loads of step j+1 are in flight while step j computes
    float2 nxt[Tree::kIn];
    load_g(0, nxt);
    for (int jb = 0; jb < steps; jb += Tree::kPeriod) {
        static_for<0, Tree::kPeriod>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int r = p_hi - j;  // z row (window end row) of this step
                float2 u[Tree::kIn];
#pragma unroll
                for (int t = 0; t < Tree::kIn; ++t) u[t] = c_scale(s, nxt[t]);
                load_g(j + 1, nxt);
                const float2 y = reduce_residues<R>(tree.template step<J>(u));
                if (c == 0 && active && r < rb) p.gz[(int64_t)r * p.nch + ch] = y;
            }
        });
    }
}

template <int M, int B, bool CPLX>
__global__ void __launch_bounds__(128) adj_row_kernel(const __grid_constant__ AdjRowParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    const int c = threadIdx.x & (R - 1);
    const int row = blockIdx.x * (blockDim.x >> B) + (threadIdx.x >> B);
    const bool active = row < p.zrows;
    const int pa = blockIdx.y * p.chunk;
    if (pa >= p.N1) return;  // uniform per block
    const int pb = min(pa + p.chunk, p.N1);
    const int p_hi = min(pb + n - 2, p.N1 - 1);
    const int steps = p_hi - pa + 1;

    const float2 *zrow = p.gz + (int64_t)(active ? row : 0) * p.P1 * n + c;

    Tree tree;
    tree.init(c, p.om64);
    for (int jb = 0; jb < steps; jb += Tree::kPeriod) {
        static_for<0, Tree::kPeriod>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = p_hi - j;
                const int q1 = p1 - (n - 1);
                float2 u[Tree::kIn];
                if (active && q1 >= 0 && q1 < p.P1) {
                    const float2 *g = zrow + (int64_t)q1 * n;
#pragma unroll
                    for (int t = 0; t < Tree::kIn; ++t) u[t] = __ldg(g + (t << B));
                } else {
#pragma unroll
                    for (int t = 0; t < Tree::kIn; ++t) u[t] = make_float2(0.f, 0.f);
                }
                const float2 y = reduce_residues<R>(tree.template step<J>(u));
                if (c == 0 && active && p1 < pb) {
                    if constexpr (CPLX)
                        reinterpret_cast<float2 *>(p.gx)[(int64_t)row * p.ld_out + p1] = y;
                    else
                        reinterpret_cast<float *>(p.gx)[(int64_t)row * p.ld_out + p1] = y.x;
                }
            }
        });
    }
}

template <int M, int B>
void adj_col_launch_mb(const AdjColParams &p, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
void adj_row_launch_mb(const AdjRowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s);

// The residue split each adjoint pass uses for a window side 2^M (registers without spills).
__host__ __device__ constexpr int adj_col_B(int M) { return M <= 4 ? (M < 1 ? M : 1) : M - 3; }
__host__ __device__ constexpr int adj_row_B(int M) { return M >= 6 ? 3 : (M < 2 ? M : 2); }

#define SWDFT_ADJ_INSTANTIATE(M_)                                                                 \
    template <>                                                                                  \
    void adj_col_launch_mb<M_, adj_col_B(M_)>(const AdjColParams &p, dim3 g, dim3 b,             \
                                              cudaStream_t s) {                                  \
        adj_col_kernel<M_, adj_col_B(M_)><<<g, b, 0, s>>>(p);                                    \
    }                                                                                            \
    template <>                                                                                  \
    void adj_row_launch_mb<M_, adj_row_B(M_)>(const AdjRowParams &p, int cplx, dim3 g, dim3 b,   \
                                              cudaStream_t s) {                                  \
        if (cplx)                                                                                \
            adj_row_kernel<M_, adj_row_B(M_), true><<<g, b, 0, s>>>(p);                          \
        else                                                                                     \
            adj_row_kernel<M_, adj_row_B(M_), false><<<g, b, 0, s>>>(p);                         \
    }

}  // namespace swdft
