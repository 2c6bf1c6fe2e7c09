// Ternary-tree passes (windows of 3, 9 or 27 along an axis; tree3_core.cuh): the row levels
// along dimension 1 and the column levels along dimension 0, laid out like the binary
// passes (tree_kernels.cuh).  z layout: z_pad rows in front (2 n0 / 3 for a ternary column
// tree: its level-0 look-back reaches 2 s_1 rows up), then rows x P1 x n1 complex64.
#include <algorithm>

#include "swdft_internal.h"
#include "tree3_core.cuh"

namespace swdft {

struct Row3Params {
    const void *x;
    int64_t ld, r_base, zrow;
    int rows, P1, chunk;
    float2 *z;
    Omega27 om;
};

struct Col3Params {
    const float2 *z;
    float2 *out;
    int64_t nch, orow;
    int rows_out, chunk, n1;
    float scale;
    Omega27 om;
};

template <bool CPLX>
__device__ __forceinline__ float2 load_x3(const char *row, int64_t i) {
    if constexpr (CPLX)
        return __ldg(reinterpret_cast<const float2 *>(row) + i);
    else
        return make_float2(__ldg(reinterpret_cast<const float *>(row) + i), 0.f);
}

// Residue split of a 3^M-point tree over three threads (M >= 1); M = 0 needs no tree.
template <int M>
struct Tree3Of {
    static constexpr bool kSplit = M >= 1;
    static constexpr int kR = kSplit ? 3 : 1;            // threads per tree
    static constexpr int kOut = kSplit ? pow3(M - 1) : 1;  // outputs per thread: k = c + 3 u
};

// Row levels: 32 rows per block, one warp per residue (3 warps; 1 when n1 = 1); lanes are
// rows.  Thread (row, c) walks window columns [qa, qb) of its row.  Each row's z values for
// consecutive windows are contiguous, so a group of kRow3Unr steps is staged in shared memory
// ([row][step][k1]) and written back row by row with consecutive threads on consecutive
// addresses.
constexpr int kRow3Unr = 6;  // a multiple of every ternary tree's period

template <int M, bool CPLX>
__global__ void __launch_bounds__(96) row_tree3_kernel(const __grid_constant__ Row3Params p) {
    constexpr int n = pow3(M);
    constexpr int OUT = Tree3Of<M>::kOut;
    constexpr int S1 = M >= 1 ? pow3(M - 1) : 0;
    constexpr int UNR = kRow3Unr;
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
    using Tree = SlidingTree3Split<(M >= 1 ? M : 1)>;
    Tree tree;
    if constexpr (M >= 1) tree.init(c, p.om);
    for (int jb = 0; jb < steps; jb += UNR) {
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = qa + j;  // window end column
                const float2 xp = load_x3<CPLX>(xrow, p1);
                float2 o[OUT];
                if constexpr (M == 0) {
                    o[0] = xp;
                } else {
                    const float2 x1 = load_x3<CPLX>(xrow, max(p1 - S1, 0));
                    const float2 x2 = load_x3<CPLX>(xrow, max(p1 - 2 * S1, 0));
                    tree.template step<J % Tree::kPeriod>(p.om.h, xp, x1, x2, o);
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
__host__ __device__ constexpr int col3_group(int M) { return M >= 3 ? 6 : 8; }  // multiple of the period
__host__ __device__ constexpr int col3_ring_rows(int M) {
    const int need = (M >= 1 ? 2 * pow3(M - 1) : 0) + 2 * col3_group(M);
    int r = 1;
    while (r < need) r <<= 1;
    return r;
}
__host__ __device__ constexpr size_t col3_smem(int M) {
    return sizeof(float2) * ((size_t)col3_ring_rows(M) * kCol3Ch + 2 * (size_t)kCol3Ch * pow3(M));
}

__device__ __forceinline__ void cp_async3_8(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}

template <int M, bool STAGED>
__global__ void __launch_bounds__(192) col_tree3_kernel(const __grid_constant__ Col3Params p) {
    constexpr int n = pow3(M);
    constexpr int R = Tree3Of<M>::kR;
    constexpr int OUT = Tree3Of<M>::kOut;
    constexpr int G = col3_group(M);
    constexpr int RD = col3_ring_rows(M);
    constexpr int S1 = M >= 1 ? pow3(M - 1) : 0;
    constexpr int W = kCol3Ch;  // ring width (lanes of the channel groups)
    using Tree = SlidingTree3Split<(M >= 1 ? M : 1)>;
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

    Tree tree;
    if constexpr (M >= 1) tree.init(c, p.om);
    int buf = 0;
    fetch(qa - 2 * S1, min(qa + G, zr_end));
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    for (int jb = 0; jb < steps; jb += G) {
        if (jb + G < steps) fetch(qa + jb + G, min(qa + jb + 2 * G, zr_end));
        static_for<0, G>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int zr = qa + j;  // z row = window end row
                const float2 xp = ring[(zr & (RD - 1)) * W + my];
                float2 o[OUT];
                if constexpr (M == 0) {
                    o[0] = xp;
                } else {
                    const float2 x1 = ring[((zr - S1) & (RD - 1)) * W + my];
                    const float2 x2 = ring[((zr - 2 * S1) & (RD - 1)) * W + my];
                    tree.template step<J % Tree::kPeriod>(p.om.h, xp, x1, x2, o);
                }
                if (j >= n - 1) {
                    if constexpr (STAGED) {
                        float2 *st = stage + buf * (W * n);
                        if (my < CH) {
#pragma unroll
                            for (int u = 0; u < OUT; ++u) st[sbase + 3 * u * p.n1] = c_scale(s, o[u]);
                        }
                        __syncthreads();
                        constexpr int NT = R * W;                 // threads per block
                        constexpr int PER = (W * n + NT - 1) / NT;  // copies per thread
#pragma unroll
                        for (int i = 0; i < PER; ++i) {
                            const int e = threadIdx.x + i * NT;
                            if (e < tile_elems) __stcs(orow + e, st[e]);
                        }
                        buf ^= 1;
                    } else if (active) {
                        // whole 32-byte sectors per window column already (n1 a multiple of 4)
#pragma unroll
                        for (int u = 0; u < OUT; ++u) __stcs(orow + sbase + 3 * u * p.n1, c_scale(s, o[u]));
                    }
                    orow += p.orow;
                }
            }
        });
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
    }
    (void)active;
}

static void fill_omega27(Omega27 &om, const float2 *om27) {
    for (int j = 0; j < kMaxN3; ++j) om.w[j] = om27[j];
    om.h = -om27[9].y;  // w_27^{-9} = w_3^{-1} = -1/2 - i sin(pi/3)
}

cudaError_t launch_row_tree3(const Row3Args &a, cudaStream_t s) {
    if (a.rows <= 0 || a.P1 <= 0) return cudaSuccess;
    if (a.m1 < 0 || a.m1 > kMaxLog3 || a.rows > INT32_MAX || a.P1 > INT32_MAX) return cudaErrorInvalidValue;
    Row3Params p;
    p.x = a.x;
    p.ld = a.ld;
    p.r_base = a.r_base;
    p.zrow = a.P1 * pow3(a.m1);
    p.rows = (int)a.rows;
    p.P1 = (int)a.P1;
    p.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.P1, a.P1);
    p.z = a.z;
    fill_omega27(p.om, a.om27);
    dim3 grid((unsigned)((a.rows + 31) / 32), (unsigned)((a.P1 + p.chunk - 1) / p.chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    const dim3 block(a.m1 >= 1 ? 96 : 32);  // a warp per residue of the split tree
    const size_t smem = sizeof(float2) * 32 * kRow3Unr * (size_t)pow3(a.m1);
    switch (a.m1 * 2 + (a.cplx ? 1 : 0)) {
        case 0: row_tree3_kernel<0, false><<<grid, block, smem, s>>>(p); break;
        case 1: row_tree3_kernel<0, true><<<grid, block, smem, s>>>(p); break;
        case 2: row_tree3_kernel<1, false><<<grid, block, smem, s>>>(p); break;
        case 3: row_tree3_kernel<1, true><<<grid, block, smem, s>>>(p); break;
        case 4: row_tree3_kernel<2, false><<<grid, block, smem, s>>>(p); break;
        case 5: row_tree3_kernel<2, true><<<grid, block, smem, s>>>(p); break;
        case 6: row_tree3_kernel<3, false><<<grid, block, smem, s>>>(p); break;
        case 7: row_tree3_kernel<3, true><<<grid, block, smem, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_col_tree3(const Col3Args &a, cudaStream_t s) {
    if (a.n1 < 1 || a.P1 < 0) return cudaErrorInvalidValue;
    const int64_t nch = a.P1 * a.n1;
    if (a.rows_out <= 0 || nch <= 0) return cudaSuccess;
    if (a.m0 < 0 || a.m0 > kMaxLog3 || a.rows_out > INT32_MAX) return cudaErrorInvalidValue;
    Col3Params p;
    p.z = a.z;
    p.out = a.out;
    p.nch = nch;
    p.orow = nch * pow3(a.m0);
    p.rows_out = (int)a.rows_out;
    p.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.rows_out, a.rows_out);
    p.n1 = a.n1;
    p.scale = a.scale;
    fill_omega27(p.om, a.om27);
    if (a.n1 > kCol3Ch) return cudaErrorInvalidValue;
    const int64_t T = std::max(1, kCol3Ch / a.n1);  // whole window columns per tile
    dim3 grid((unsigned)((a.P1 + T - 1) / T), (unsigned)((a.rows_out + p.chunk - 1) / p.chunk));
    if (grid.y > 65535 || grid.x == 0) return cudaErrorInvalidValue;
    const size_t smem = col3_smem(a.m0);
    const dim3 block(a.m0 >= 1 ? 3 * kCol3Ch : kCol3Ch);  // a warp per (residue, 32 channels)
    const bool staged = a.n1 % 4 != 0;
    switch (a.m0 * 2 + (staged ? 1 : 0)) {
        case 0: col_tree3_kernel<0, false><<<grid, block, smem, s>>>(p); break;
        case 1: col_tree3_kernel<0, true><<<grid, block, smem, s>>>(p); break;
        case 2: col_tree3_kernel<1, false><<<grid, block, smem, s>>>(p); break;
        case 3: col_tree3_kernel<1, true><<<grid, block, smem, s>>>(p); break;
        case 4: col_tree3_kernel<2, false><<<grid, block, smem, s>>>(p); break;
        case 5: col_tree3_kernel<2, true><<<grid, block, smem, s>>>(p); break;
        case 6: col_tree3_kernel<3, false><<<grid, block, smem, s>>>(p); break;
        case 7: col_tree3_kernel<3, true><<<grid, block, smem, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
