// Ternary and mixed-radix tree passes (windows of 3^b 2^a samples along an axis, b >= 1,
// at most 64; tree3_core.cuh): the row levels along dimension 1 and the column levels along
// dimension 0, laid out like the binary passes (tree_kernels.cuh).  z layout: z_pad rows in
// front (2 n0 / 3 for such a column tree, the reach of its level-0 look-back; walks that
// start 2 s_1 steps in, as these do, never read them), then rows x P1 x n1 complex64.  Kernels are templated on (B3, A2), n = 3^B3 2^A2; (0, 0) is the
// window of one sample (no tree).
#pragma once

#include <algorithm>

#include "sm100_ptx.cuh"
#include "swdft_internal.h"
#include "tree3_core.cuh"

namespace swdft {

struct Row3Params {
    const void *x;
    int64_t ld, r_base, zrow;
    int rows, P1, chunk;
    float2 *z;
    OmegaN om;
};

struct Col3Params {
    const float2 *z;
    float2 *out;
    int64_t nch, orow;
    int rows_out, chunk, n1;
    float scale;
    OmegaN om;
};

template <bool CPLX>
__device__ __forceinline__ float2 load_x3(const char *row, int64_t i) {
    if constexpr (CPLX)
        return __ldg(reinterpret_cast<const float2 *>(row) + i);
    else
        return make_float2(__ldg(reinterpret_cast<const float *>(row) + i), 0.f);
}

// Residue split of an n-point tree over three threads (B3 >= 1); n = 1 needs no tree.
template <int B3, int A2>
struct TreeMOf {
    static constexpr bool kSplit = B3 >= 1;
    static constexpr int kN = mixed_n(B3, A2);
    static constexpr int kR = kSplit ? 3 : 1;            // threads per tree
    static constexpr int kOut = kSplit ? kN / 3 : 1;     // outputs per thread: k = c + 3 u
    static constexpr int kS1 = kSplit ? kN / 3 : 0;
    using Tree = SlidingTreeMixed<(B3 >= 1 ? B3 : 1), (B3 >= 1 ? A2 : 0)>;
    static constexpr int kPeriod = kSplit ? Tree::kPeriod : 1;
};

// Steps per unrolled group of the row pass (a multiple of the tree's period, at least 6).
__host__ __device__ constexpr int row3_unr(int period) {
    return period <= 6 && 6 % period == 0 ? 6 : (period <= 8 && 8 % period == 0 ? 8 : 12);
}

// Row levels: 32 rows per block, one warp per residue (3 warps; 1 when n1 = 1); lanes are
// rows.  Thread (row, c) walks window columns [qa, qb) of its row.  Each row's z values for
// consecutive windows are contiguous, so a group of row3_unr steps is staged in shared memory
// ([row][step][k1]) and written back row by row with consecutive threads on consecutive
// addresses.
template <int B3, int A2, bool CPLX>
__global__ void __launch_bounds__(96) row_tree3_kernel(const __grid_constant__ Row3Params p) {
    using Of = TreeMOf<B3, A2>;
    constexpr int n = Of::kN;
    constexpr int OUT = Of::kOut;
    constexpr int S1 = Of::kS1;
    constexpr int UNR = row3_unr(Of::kPeriod);
    extern __shared__ float2 stage[];  // 32 x UNR x n
    const int c = threadIdx.x >> 5;    // residue: warp-uniform
    const int lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * 32;
    const int row = row0 + lane;
    const bool live = row < p.rows;
    const int nrows = min(32, p.rows - row0);
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.P1) return;  // uniform per block
    const int qb = min(qa + p.chunk, p.P1);
    const int steps = (qb - qa) + (n - 1);
    const char *xrow = reinterpret_cast<const char *>(p.x) +
                       (p.r_base + (live ? row : row0)) * p.ld * (int64_t)(CPLX ? sizeof(float2) : sizeof(float));
    using Tree = typename Of::Tree;
    Tree tree;
    if constexpr (Of::kSplit) tree.init(c, p.om);
    // The walk starts at step 2 s_1 (= 2n/3): level 1 reads level 0 s_1 and 2 s_1 back from
    // memory and the FIFOs of levels 1 .. L-1 hold n - 1 - 2 s_1 steps, so the first stored
    // output (step n - 1) needs level 1 from step 2 s_1 on.  2 s_1 is a multiple of the unroll
    // period.
    static_assert(!Of::kSplit || (2 * S1) % Of::kPeriod == 0, "the walk starts on a whole period");
    for (int jb = 2 * S1; jb < steps; jb += UNR) {
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = qa + j;  // window end column
                const float2 xp = load_x3<CPLX>(xrow, p1);
                float2 o[OUT];
                if constexpr (!Of::kSplit) {
                    o[0] = xp;
                } else {
                    const float2 x1 = load_x3<CPLX>(xrow, max(p1 - S1, 0));
                    const float2 x2 = load_x3<CPLX>(xrow, max(p1 - 2 * S1, 0));
                    tree.template step<J % Tree::kPeriod>(p.om.h, 1.f, xp, x1, x2, o);
                }
                if (j >= n - 1) {
#pragma unroll
                    for (int u = 0; u < OUT; ++u) stage[(lane * UNR + J) * n + c + 3 * u] = o[u];
                }
            }
        });
        // outputs of this group: steps [max(jb, n-1), min(jb + UNR, steps)), windows from q
        const int j0 = max(jb, n - 1), j1 = min(jb + UNR, steps);
        __syncthreads();
        if (j1 > j0) {
            const int run = (j1 - j0) * n;           // contiguous values per row
            const int q = qa + j0 - (n - 1);         // first window of the run
            const int sofs = (j0 - jb) * n;          // its offset in a row's stage
            float2 *zq = p.z + (int64_t)row0 * p.zrow + (int64_t)q * n;
            const float2 *sq = stage + sofs;
            for (int r = 0; r < nrows; ++r) {
                for (int k = threadIdx.x; k < run; k += blockDim.x) zq[k] = sq[k];
                zq += p.zrow;
                sq += UNR * n;
            }
        }
        __syncthreads();
    }
}

// Column levels: a block takes T = 64 / n1 whole window columns q1 (CH = T n1 <= 64
// channels (q1, k1) of z, any n1) and one chunk of window rows; one warp per (residue,
// 32-channel group).  The tile's z rows reach a shared-memory ring one group ahead
// (cp.async); the level-0 look-backs 2 s_1 rows up come from the same ring, and all three
// residue warps of a channel group read the same staged rows.  For every window row the
// tile's outputs out[q0][q1 .. q1+T-1][k0][k1] are one contiguous run of T n0 n1 values;
// when n1 is not a multiple of 4 (window columns that are not whole 32-byte sectors) they
// are staged in shared memory (double-buffered) and written back with consecutive threads
// on consecutive addresses; otherwise each thread stores its own outputs.
constexpr int kCol3Ch = 64;
// rows per staged group: a multiple of the tree's period, at least 6
__host__ __device__ constexpr int col3_group(int period) {
    return period <= 8 && 8 % period == 0 ? 8 : (period == 6 ? 6 : 12);
}
__host__ __device__ constexpr int col3_ring_rows(int n, int period) {
    const int need = (n >= 3 ? 2 * (n / 3) : 0) + 2 * col3_group(period);
    int r = 1;
    while (r < need) r <<= 1;
    return r;
}
__host__ __device__ constexpr size_t col3_smem(int n, int period) {
    return sizeof(float2) * ((size_t)col3_ring_rows(n, period) * kCol3Ch + 2 * (size_t)kCol3Ch * n);
}

// Bulk copy of `bytes` (a multiple of 16) from shared to global memory (both 16-byte aligned),
// issued by one thread, with an evict-first L2 policy (the output is written once and should
// not push z out of L2); read_wait() returns once every copy this thread issued has finished
// reading shared memory, all_wait() once they are complete.
__device__ __forceinline__ void bulk_store_evict_first(void *gmem, const void *smem, uint32_t bytes) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;\n" ::"l"(gmem),
                 "r"(smem_u32(smem)), "r"(bytes), "l"(pol)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_store_read_wait() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_store_all_wait() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async3_8(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}

template <int B3, int A2, bool STAGED>
__global__ void __launch_bounds__(192) col_tree3_kernel(const __grid_constant__ Col3Params p) {
    using Of = TreeMOf<B3, A2>;
    constexpr int n = Of::kN;
    constexpr int R = Of::kR;
    constexpr int OUT = Of::kOut;
    constexpr int G = col3_group(Of::kPeriod);
    constexpr int RD = col3_ring_rows(n, Of::kPeriod);
    constexpr int S1 = Of::kS1;
    constexpr int W = kCol3Ch;  // ring width (lanes of the channel groups)
    using Tree = typename Of::Tree;
    extern __shared__ float2 smem3[];
    float2 *ring = smem3;                // RD x W
    float2 *stage = smem3 + RD * W;      // 2 x (CH n0)
    const int T = max(1, W / p.n1);      // whole window columns per tile
    const int CH = T * p.n1;             // channels per tile
    const int warp = threadIdx.x >> 5;
    const int c = warp % R;                              // residue (warp-uniform)
    const int my = (warp / R) * 32 + (threadIdx.x & 31);  // channel within the tile
    const int64_t q1_0 = (int64_t)blockIdx.x * T;
    const int64_t ch0 = q1_0 * p.n1;
    const int64_t ch = ch0 + my;
    const bool active = my < CH && ch < p.nch;
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.rows_out) return;  // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const int steps = (qb - qa) + (n - 1);
    const int zr_end = qb + n - 1;  // one past the last z row used
    const int tile_elems = (int)(min((int64_t)T, p.nch / p.n1 - q1_0) * n) * p.n1;  // valid outputs per window row
    const int q1l = my / p.n1, k1 = my - q1l * p.n1;
    const int sbase = q1l * n * p.n1 + c * p.n1 + k1;  // this thread's first staged output
    float2 *orow = p.out + (int64_t)qa * p.orow + q1_0 * n * p.n1;
    const float s = p.scale;
    // The staged run of a window row goes out as one bulk copy when it starts 16-byte aligned
    // and holds an even number of values (output rows of an even length, an even first value):
    // the stage buffers start on 16 bytes (ring and buffers are multiples of 64 values).
    // Otherwise every thread copies its share of the run.
    const bool bulk = STAGED && p.orow % 2 == 0 && (q1_0 * n * p.n1) % 2 == 0 && tile_elems % 2 == 0 &&
                      reinterpret_cast<uintptr_t>(p.out) % 16 == 0;

    auto fetch = [&](int r_lo, int r_hi) {
        const int total = (r_hi - r_lo) * CH;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int rr = r_lo + e / CH;
            const int cc = e - (e / CH) * CH;
            const bool ok = ch0 + cc < p.nch;
            cp_async3_8(&ring[(rr & (RD - 1)) * W + cc], p.z + (int64_t)rr * p.nch + (ok ? ch0 + cc : 0), ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // the scale is folded into the tree's level 1 (an n0 = 1 window, with no tree, scales here)
    Tree tree;
    if constexpr (Of::kSplit) tree.init(c, p.om, s);
    int buf = 0;
    // the walk starts at step 2 s_1, as in the row pass: its look-backs start at row qa
    fetch(qa, min(qa + 2 * S1 + G, zr_end));
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    static_assert(!Of::kSplit || (2 * S1) % Of::kPeriod == 0, "the walk starts on a whole period");
    for (int jb = 2 * S1; jb < steps; jb += G) {
        if (jb + G < steps) fetch(qa + jb + G, min(qa + jb + 2 * G, zr_end));
        static_for<0, G>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int zr = qa + j;  // z row = window end row
                const float2 xp = ring[(zr & (RD - 1)) * W + my];
                float2 o[OUT];
                if constexpr (!Of::kSplit) {
                    o[0] = c_scale(s, xp);
                } else {
                    const float2 x1 = ring[((zr - S1) & (RD - 1)) * W + my];
                    const float2 x2 = ring[((zr - 2 * S1) & (RD - 1)) * W + my];
                    tree.template step<J % Tree::kPeriod>(p.om.h, s, xp, x1, x2, o);
                }
                if (j >= n - 1) {
                    if constexpr (STAGED) {
                        float2 *st = stage + buf * (W * n);
                        if (my < CH) {
#pragma unroll
                            for (int u = 0; u < OUT; ++u) st[sbase + 3 * u * p.n1] = o[u];
                        }
                        if (bulk) {
                            // this thread's stores are made visible to the bulk copy; thread 0
                            // waits until the previous row's copy has read the other buffer
                            // (the one the next row writes) before the barrier publishes it
                            fence_proxy_async_smem();
                            if (threadIdx.x == 0) bulk_store_read_wait();
                        }
                        __syncthreads();
                        constexpr int NT = R * W;                 // threads per block
                        if (bulk) {
                            if (threadIdx.x == 0) bulk_store_evict_first(orow, st, (uint32_t)tile_elems * 8u);
                        } else {
                            constexpr int PER = (W * n + NT - 1) / NT;  // copies per thread
#pragma unroll
                            for (int i = 0; i < PER; ++i) {
                                const int e = threadIdx.x + i * NT;
                                if (e < tile_elems) __stcs(orow + e, st[e]);
                            }
                        }
                        buf ^= 1;
                    } else if (active) {
                        // whole 32-byte sectors per window column already (n1 a multiple of 4)
#pragma unroll
                        for (int u = 0; u < OUT; ++u) __stcs(orow + sbase + 3 * u * p.n1, o[u]);
                    }
                    orow += p.orow;
                }
            }
        });
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
    }
    if (bulk && threadIdx.x == 0) bulk_store_all_wait();  // the stage stays valid until read
    (void)active;
}

// Window shapes built: n = 1, 3, 6, 12, 24, 48, 9, 18, 36, 27, 54 as (B3, A2).
#define SWDFT_MIXED_CASES(F) \
    F(0, 0) F(1, 0) F(1, 1) F(1, 2) F(1, 3) F(1, 4) F(2, 0) F(2, 1) F(2, 2) F(3, 0) F(3, 1)

template <int B3, int A2>
void row3_launch_ba(const Row3Params &p, int cplx, dim3 g, dim3 b, cudaStream_t s);
template <int B3, int A2>
void col3_launch_ba(const Col3Params &p, int staged, dim3 g, dim3 b, cudaStream_t s);

// dynamic shared memory above 48 KB is opted into once per instantiation
#define SWDFT_ROW3_INSTANTIATE(B3_, A2_)                                                            \
    template <>                                                                                    \
    void row3_launch_ba<B3_, A2_>(const Row3Params &p, int cplx, dim3 g, dim3 b, cudaStream_t s) {  \
        using Of = TreeMOf<B3_, A2_>;                                                              \
        constexpr size_t smem = sizeof(float2) * 32 * row3_unr(Of::kPeriod) * Of::kN;              \
        static const bool attr = smem <= 48 * 1024 ||                                              \
            (cudaFuncSetAttribute(row_tree3_kernel<B3_, A2_, true>,                                \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==       \
                 cudaSuccess &&                                                                    \
             cudaFuncSetAttribute(row_tree3_kernel<B3_, A2_, false>,                               \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==       \
                 cudaSuccess);                                                                     \
        (void)attr;                                                                                \
        if (cplx)                                                                                  \
            row_tree3_kernel<B3_, A2_, true><<<g, b, smem, s>>>(p);                                \
        else                                                                                       \
            row_tree3_kernel<B3_, A2_, false><<<g, b, smem, s>>>(p);                               \
    }

#define SWDFT_COL3_INSTANTIATE(B3_, A2_)                                                            \
    template <>                                                                                    \
    void col3_launch_ba<B3_, A2_>(const Col3Params &p, int staged, dim3 g, dim3 b, cudaStream_t s) { \
        using Of = TreeMOf<B3_, A2_>;                                                              \
        constexpr size_t smem = col3_smem(Of::kN, Of::kPeriod);                                    \
        static const bool attr = smem <= 48 * 1024 ||                                              \
            (cudaFuncSetAttribute(col_tree3_kernel<B3_, A2_, true>,                                \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==       \
                 cudaSuccess &&                                                                    \
             cudaFuncSetAttribute(col_tree3_kernel<B3_, A2_, false>,                               \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==       \
                 cudaSuccess);                                                                     \
        (void)attr;                                                                                \
        if (staged)                                                                                \
            col_tree3_kernel<B3_, A2_, true><<<g, b, smem, s>>>(p);                                \
        else                                                                                       \
            col_tree3_kernel<B3_, A2_, false><<<g, b, smem, s>>>(p);                               \
    }

}  // namespace swdft
