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
// adj_col splits the work by WINDOW rows: chunk i takes windows q0 in [qa, qb) and reads
// those rows of G exactly once (G is the large operand: n0 times gz).  Its outputs cover z
// rows [qa, qb + n0 - 2]; rows >= qb are shared with chunk i+1, so chunk i writes them to a
// side buffer, side[i][r - qb][ch] (n0-1 rows per chunk boundary), and adj_row adds them to
// gz rows [qb, qb + n0 - 2] as it reads them.  Every gz row is written exactly once.
//
// Lanes hold (residue c in the low B bits, channel or row above): the 2^B partials of one
// output are reduced with shuffles and lane c = 0 stores.  G is read once, coalesced: for a
// fixed node t the lanes of one residue read consecutive k1 of one k0 row.
#pragma once

#include <cstdint>

#include "swdft_internal.h"
#include "adjoint_core.cuh"

namespace swdft {

// Per array (grid z) pointers: arrays of one shape share a launch.
struct AdjColParams {
    const float2 *G[kAdjZ];   // rows_out x P1 x n0 x n1
    float2 *gz[kAdjZ];        // (rows_out + n0 - 1) x P1 x n1
    float2 *side[kAdjZ];      // (chunks - 1) x (n0 - 1) x P1 x n1: rows shared with the next chunk
    int64_t nch;       // P1 * n1
    int rows_out;      // window rows of G
    int chunk;         // window rows per chunk (walked with n0 - 1 more drain steps)
    int m1;
    float scale;
    float2 om64[kMaxN];  // w_64^{-j}: every power-of-two length's twiddles
};

struct AdjRowParams {
    const float2 *gz[kAdjZ];    // zrows x P1 x n1
    const float2 *side[kAdjZ];  // adj_col's side buffers (see AdjColParams), or null
    void *gx[kAdjZ];            // zrows rows of N1 elements (row stride ld_out)
    int64_t ld_out;
    int zrows;
    int N1, P1;
    int chunk;         // output columns per thread (plus n1 - 1 warm-up steps)
    int col_chunk;     // adj_col's window rows per chunk
    int rows_out;      // window rows of G
    int n0m1;          // n0 - 1: side rows per chunk boundary
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

// G staging for adj_col: a block's channels (128 >> B consecutive (q1, k1)) need, per window
// row, n0 x (128 >> B) values (8 KB for every n0 >= 16 with the built splits).  They are
// copied into a shared-memory ring by cp.async in groups of kAdjGroup steps, one group ahead
// of use (a 32 KB ring, so that five blocks of 128 threads fit an SM), laid out [step][k0][channel] so the lanes of one residue read consecutive words.
constexpr int kAdjGroup = 2;
__host__ __device__ constexpr int adj_col_channels(int B) { return 128 >> B; }
__host__ __device__ constexpr size_t adj_col_smem(int M, int B) {
    return sizeof(float2) * 2 * kAdjGroup * (size_t(1) << M) * adj_col_channels(B);
}

__device__ __forceinline__ void adj_cp_async_8(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void adj_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void adj_cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void adj_cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int M, int B>
__global__ void __launch_bounds__(128) adj_col_kernel(const __grid_constant__ AdjColParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    constexpr int CH = adj_col_channels(B);
    constexpr int GS = kAdjGroup;
    // steps per unrolled iteration: a multiple of both the tree's period and the group
    constexpr int UNR = Tree::kPeriod > GS ? Tree::kPeriod : GS;
    constexpr int STEP = n * CH;  // staged values per step
    extern __shared__ float2 sg[];  // [2][GS][n][CH]

    const int c = threadIdx.x & (R - 1);
    const int chl = threadIdx.x >> B;  // this thread's channel within the block
    const int64_t ch0 = (int64_t)blockIdx.x * CH;
    const int64_t ch = ch0 + chl;
    const bool active = ch < p.nch;
    const int qa = blockIdx.y * p.chunk;  // windows [qa, qb) of this chunk
    if (qa >= p.rows_out) return;         // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const bool last = qb == p.rows_out;
    const int p_hi = qb + n - 2;          // end row of the chunk's top window
    const int nwin = qb - qa;
    const int steps = nwin + n - 1;       // down to z row qa

    const int n1 = 1 << p.m1;
    const int64_t grow = p.nch * n;  // elements per window row of G
    const float s = p.scale;
    const float2 *G = p.G[blockIdx.z];
    float2 *gz = p.gz[blockIdx.z];
    float2 *side = p.side[blockIdx.z] + (int64_t)blockIdx.y * (n - 1) * p.nch + ch;

    // copy the G rows of steps [j0, j0 + GS) that exist (window row qb - 1 - j) into buffer b.
    // The block has 128 = R * CH threads, so copying thread i always takes channel i mod CH
    // and the k0 = i / CH + R * t, t < n / R, of every step: one base address per thread.
    const int cl_f = threadIdx.x & (CH - 1);
    const int k0_f = threadIdx.x / CH;
    const int64_t cg_f = ch0 + cl_f;
    const bool ok_f = cg_f < p.nch;
    const float2 *gsrc = G + (ok_f ? ((cg_f >> p.m1) * n + k0_f) * n1 + (cg_f & (n1 - 1)) : 0);
    const int64_t kstep = (int64_t)R * n1;  // global distance between a thread's k0 values
    auto fetch = [&](int j0, int b) {
        const int cnt = min(GS, nwin - j0);
        float2 *dst = sg + b * GS * STEP + k0_f * CH + cl_f;
        const float2 *src = gsrc + (int64_t)(qb - 1 - j0) * grow;
        for (int st = 0; st < cnt; ++st) {
#pragma unroll
            for (int t = 0; t < n / R; ++t) adj_cp_async_8(dst + t * R * CH, src + t * kstep, ok_f);
            dst += STEP;
            src -= grow;
        }
        adj_cp_async_commit();
    };

    Tree tree;
    tree.init(c, p.om64);
    if (nwin > 0) fetch(0, 0);
    for (int jb = 0; jb < steps; jb += UNR) {
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if constexpr (J % GS == 0) {
                // group j / GS: start fetching the next one, then wait for this one
                const int g = j / GS;
                if (j + GS < nwin) {
                    fetch(j + GS, (g + 1) & 1);
                    adj_cp_async_wait_1();
                } else {
                    adj_cp_async_wait_0();
                }
                __syncthreads();
            }
            if (j < steps) {
                const int r = p_hi - j;  // z row (window end row) of this step
                float2 u[Tree::kIn];
                if (j < nwin) {
                    const float2 *src = sg + (((j / GS) & 1) * GS + (J % GS)) * STEP + chl;
#pragma unroll
                    for (int t = 0; t < Tree::kIn; ++t) u[t] = src[(c + R * t) * CH];
                } else {
#pragma unroll
                    for (int t = 0; t < Tree::kIn; ++t) u[t] = make_float2(0.f, 0.f);
                }
                // the transposed tree is linear: scale its output instead of its n0 inputs
                const float2 y = c_scale(s, reduce_residues<R>(tree.template step<J>(u)));
                if (c == 0 && active) {
                    if (r >= qb && !last)
                        side[(int64_t)(r - qb) * p.nch] = y;
                    else
                        gz[(int64_t)r * p.nch + ch] = y;
                }
            }
            if constexpr (J % GS == GS - 1) __syncthreads();  // the buffer is refilled next group
        });
    }
}

template <int M, int B, bool CPLX>
__global__ void __launch_bounds__(128) adj_row_kernel(const __grid_constant__ AdjRowParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    // gz loads issued PF steps ahead (a divisor of the unroll period; two for the larger
    // trees, whose registers are already mostly taken by their FIFOs)
    constexpr int PF = M >= 5 ? 2 : (Tree::kPeriod >= 4 ? 4 : Tree::kPeriod);
    const int c = threadIdx.x & (R - 1);
    const int row = blockIdx.x * (blockDim.x >> B) + (threadIdx.x >> B);
    const bool active = row < p.zrows;
    const int pa = blockIdx.y * p.chunk;
    if (pa >= p.N1) return;  // uniform per block
    const int pb = min(pa + p.chunk, p.N1);
    const int p_hi = min(pb + n - 2, p.N1 - 1);
    const int steps = p_hi - pa + 1;

    const int64_t rowlen = (int64_t)p.P1 * n;
    const float2 *zrow = p.gz[blockIdx.z] + (int64_t)(active ? row : 0) * rowlen + c;
    const float2 *sidez = p.side[blockIdx.z];
    void *gx = p.gx[blockIdx.z];
    // the part of this z row adj_col's previous chunk left in its side buffer, if any
    const float2 *srow = nullptr;
    if (sidez != nullptr && active && p.n0m1 > 0) {
        const int i = row / p.col_chunk;  // chunk whose windows start at row i * col_chunk
        const int off = row - i * p.col_chunk;
        if (i >= 1 && i * p.col_chunk < p.rows_out && off < p.n0m1)
            srow = sidez + ((int64_t)(i - 1) * p.n0m1 + off) * rowlen + c;
    }

    auto load_z = [&](int j, float2 (&u)[Tree::kIn]) {
        const int q1 = p_hi - j - (n - 1);
        if (active && j < steps && q1 >= 0 && q1 < p.P1) {
            const float2 *g = zrow + (int64_t)q1 * n;
#pragma unroll
            for (int t = 0; t < Tree::kIn; ++t) u[t] = __ldg(g + (t << B));
            if (srow != nullptr) {
                const float2 *h = srow + (int64_t)q1 * n;
#pragma unroll
                for (int t = 0; t < Tree::kIn; ++t) u[t] = c_add(u[t], __ldg(h + (t << B)));
            }
        } else {
#pragma unroll
            for (int t = 0; t < Tree::kIn; ++t) u[t] = make_float2(0.f, 0.f);
        }
    };

    Tree tree;
    tree.init(c, p.om64);
    float2 buf[PF][Tree::kIn];
#pragma unroll
    for (int d = 0; d < PF; ++d) load_z(d, buf[d]);
    for (int jb = 0; jb < steps; jb += Tree::kPeriod) {
        static_for<0, Tree::kPeriod>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            constexpr int SL = J % PF;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = p_hi - j;
                float2 u[Tree::kIn];
#pragma unroll
                for (int t = 0; t < Tree::kIn; ++t) u[t] = buf[SL][t];
                load_z(j + PF, buf[SL]);
                const float2 y = reduce_residues<R>(tree.template step<J>(u));
                if (c == 0 && active && p1 < pb) {
                    if constexpr (CPLX)
                        reinterpret_cast<float2 *>(gx)[(int64_t)row * p.ld_out + p1] = y;
                    else
                        reinterpret_cast<float *>(gx)[(int64_t)row * p.ld_out + p1] = y.x;
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
__host__ __device__ constexpr int adj_row_B(int M) { return M >= 4 ? 3 : (M < 2 ? M : 2); }

#define SWDFT_ADJ_INSTANTIATE(M_)                                                                 \
    template <>                                                                                  \
    void adj_col_launch_mb<M_, adj_col_B(M_)>(const AdjColParams &p, dim3 g, dim3 b,             \
                                              cudaStream_t s) {                                  \
        constexpr size_t smem = adj_col_smem(M_, adj_col_B(M_));                                 \
        static const bool attr_set = smem <= 48 * 1024 ||                                        \
            cudaFuncSetAttribute(adj_col_kernel<M_, adj_col_B(M_)>,                              \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==      \
                cudaSuccess;                                                                     \
        (void)attr_set;                                                                          \
        adj_col_kernel<M_, adj_col_B(M_)><<<g, b, smem, s>>>(p);                                 \
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
