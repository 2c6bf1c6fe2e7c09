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
// side buffer, side[i][r - qb][ch] (n0-1 rows per chunk boundary), and adj_fold then adds
// them to gz rows [qb, qb + n0 - 2].  No atomics: the result is deterministic.  adj_row
// stages gz rows through shared memory, GS steps at a time.
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
    void *gx[kAdjZ];            // zrows rows of N1 elements (row stride ld_out)
    int64_t ld_out;
    int zrows;
    int N1, P1;
    int chunk;         // output columns per thread (plus n1 - 1 warm-up steps)
    float2 om64[kMaxN];  // w_64^{-j}: every power-of-two length's twiddles
};

struct AdjFoldParams {
    float2 *gz[kAdjZ];
    const float2 *side[kAdjZ];
    int64_t nch;       // P1 * n1
    int64_t per_row;   // (n0 - 1) * nch: side values per chunk boundary
    int64_t total;     // (chunks - 1) * per_row
    int chunk;         // window rows per adj_col chunk
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

// G is read once: its lines are marked evict-first in L2, so that the gz rows this pass
// writes (n0 times smaller) are still in L2 when adj_row reads them.
__device__ __forceinline__ uint64_t adj_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void adj_cp_async_8(void *smem, const void *gmem, bool valid, uint64_t pol) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2, %3;\n" ::"r"(dst), "l"(gmem),
                 "r"(valid ? 8 : 0), "l"(pol)
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
    const uint64_t pol = adj_policy_evict_first();
    auto fetch = [&](int j0, int b) {
        const int cnt = min(GS, nwin - j0);
        float2 *dst = sg + b * GS * STEP + k0_f * CH + cl_f;
        const float2 *src = gsrc + (int64_t)(qb - 1 - j0) * grow;
        for (int st = 0; st < cnt; ++st) {
#pragma unroll
            for (int t = 0; t < n / R; ++t) adj_cp_async_8(dst + t * R * CH, src + t * kstep, ok_f, pol);
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

// gz staging for adj_row: a block's rows (128 >> B of them) need n1 values per row per step,
// consecutive steps reading consecutive (descending) q1, so GS steps of one row are one
// contiguous run of GS * n1 values.  Groups of GS steps (16 KB per block) are copied by
// cp.async into a double-buffered ring, one group ahead of use, 16 bytes per copy (8 for
// n1 = 1); rows are padded by R values so that the 2^B lanes of 32 / 2^B rows hit distinct banks.
template <int M, int B>
struct AdjRowStage {
    static constexpr int R = 1 << B;
    static constexpr int kRows = 128 >> B;  // rows per block
    static constexpr int kN = 1 << M;
    static constexpr int kGS0 = 2048 / (kRows * kN);
    static constexpr int kGS = kGS0 < 1 ? 1 : (kGS0 > 16 ? 16 : kGS0);  // steps per group
    static constexpr int kRow = kGS * kN + R;    // staged values per row (padded)
    static constexpr int kPiece = kN >= 2 ? 2 : 1;  // values per copy
    static constexpr int kPerRow = kGS * kN / kPiece;  // copies per row per group
    static constexpr size_t kBytes = sizeof(float2) * 2 * kRows * kRow;
    static_assert(kPerRow <= 128 && 128 % kPerRow == 0, "copies of a group must tile the block");
    static_assert(kPiece == 1 || kRow % 2 == 0, "16-byte copies need 16-byte aligned rows");
};

template <int M, int B>
__host__ __device__ constexpr size_t adj_row_smem() { return AdjRowStage<M, B>::kBytes; }

__device__ __forceinline__ void adj_cp_async_16(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void adj_cp_async_8_plain(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}

template <int M, int B, bool CPLX>
__global__ void __launch_bounds__(128) adj_row_kernel(const __grid_constant__ AdjRowParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    using St = AdjRowStage<M, B>;
    constexpr int R = St::R;
    constexpr int n = St::kN;
    constexpr int GS = St::kGS;
    constexpr int UNR = Tree::kPeriod > GS ? Tree::kPeriod : GS;
    extern __shared__ float2 sz[];  // [2][kRows][kRow]

    const int c = threadIdx.x & (R - 1);
    const int rl = threadIdx.x >> B;  // this thread's row within the block
    const int row0 = blockIdx.x * St::kRows;
    const int row = row0 + rl;
    const bool active = row < p.zrows;
    const int pa = blockIdx.y * p.chunk;
    if (pa >= p.N1) return;  // uniform per block
    const int pb = min(pa + p.chunk, p.N1);
    const int p_hi = min(pb + n - 2, p.N1 - 1);
    const int steps = p_hi - pa + 1;
    const int q1_top = p_hi - (n - 1);  // q1 of step 0; step j reads q1_top - j

    const int64_t rowlen = (int64_t)p.P1 * n;
    const float2 *gz = p.gz[blockIdx.z];
    void *gx = p.gx[blockIdx.z];

    // copying thread i always takes piece i mod kPerRow of rows i / kPerRow + t * (128 / kPerRow)
    constexpr int kRowStep = 128 / St::kPerRow;
    constexpr int kCopies = St::kRows / kRowStep;
    const int off_f = (threadIdx.x % St::kPerRow) * St::kPiece;  // value offset in the group's run
    const int rl_f = threadIdx.x / St::kPerRow;
    const int dq_f = off_f / n;  // q1 of this piece relative to the group's lowest q1
    auto fetch = [&](int j0, int b) {
        const int q1lo = q1_top - j0 - (GS - 1);
        const int q = q1lo + dq_f;
        const bool qok = q >= 0 && q < p.P1;
        const int64_t goff = (int64_t)q1lo * n + off_f;
        float2 *dst = sz + (b * St::kRows + rl_f) * St::kRow + off_f;
#pragma unroll
        for (int t = 0; t < kCopies; ++t) {
            const int r = row0 + rl_f + t * kRowStep;
            const bool ok = qok && r < p.zrows;
            const float2 *src = ok ? gz + (int64_t)r * rowlen + goff : gz;
            if constexpr (St::kPiece == 2)
                adj_cp_async_16(dst + t * kRowStep * St::kRow, src, ok);
            else
                adj_cp_async_8_plain(dst + t * kRowStep * St::kRow, src, ok);
        }
        adj_cp_async_commit();
    };

    Tree tree;
    tree.init(c, p.om64);
    fetch(0, 0);
    for (int jb = 0; jb < steps; jb += UNR) {
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if constexpr (J % GS == 0) {
                if (j + GS < steps) {
                    fetch(j + GS, ((j / GS) + 1) & 1);
                    adj_cp_async_wait_1();
                } else {
                    adj_cp_async_wait_0();
                }
                __syncthreads();
            }
            if (j < steps) {
                const int p1 = p_hi - j;
                const float2 *src = sz + (((j / GS) & 1) * St::kRows + rl) * St::kRow + (GS - 1 - (J % GS)) * n + c;
                float2 u[Tree::kIn];
#pragma unroll
                for (int t = 0; t < Tree::kIn; ++t) u[t] = src[t * R];
                const float2 y = reduce_residues<R>(tree.template step<J>(u));
                if (c == 0 && active && p1 < pb) {
                    if constexpr (CPLX)
                        reinterpret_cast<float2 *>(gx)[(int64_t)row * p.ld_out + p1] = y;
                    else
                        reinterpret_cast<float *>(gx)[(int64_t)row * p.ld_out + p1] = y.x;
                }
            }
            if constexpr (J % GS == GS - 1) __syncthreads();  // the buffer is refilled next group
        });
    }
}

template <int M, int B>
void adj_col_launch_mb(const AdjColParams &p, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
void adj_row_launch_mb(const AdjRowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
int adj_row_bps_mb(int cplx);  // resident 128-thread blocks per SM (occupancy API; 0 on error)

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
        constexpr size_t smem = adj_row_smem<M_, adj_row_B(M_)>();                               \
        static const bool attr_set =                                                             \
            smem <= 48 * 1024 ||                                                                 \
            (cudaFuncSetAttribute(adj_row_kernel<M_, adj_row_B(M_), true>,                       \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==     \
                 cudaSuccess &&                                                                  \
             cudaFuncSetAttribute(adj_row_kernel<M_, adj_row_B(M_), false>,                      \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==     \
                 cudaSuccess);                                                                   \
        (void)attr_set;                                                                          \
        if (cplx)                                                                                \
            adj_row_kernel<M_, adj_row_B(M_), true><<<g, b, smem, s>>>(p);                       \
        else                                                                                     \
            adj_row_kernel<M_, adj_row_B(M_), false><<<g, b, smem, s>>>(p);                      \
    }                                                                                            \
    template <>                                                                                  \
    int adj_row_bps_mb<M_, adj_row_B(M_)>(int cplx) {                                            \
        constexpr size_t smem = adj_row_smem<M_, adj_row_B(M_)>();                               \
        int nb = 0;                                                                              \
        cudaError_t e = cplx ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                                   &nb, adj_row_kernel<M_, adj_row_B(M_), true>, 128, smem)      \
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                                   &nb, adj_row_kernel<M_, adj_row_B(M_), false>, 128, smem);    \
        return e == cudaSuccess ? nb : 0;                                                        \
    }

}  // namespace swdft
