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

// Thread = (row, chunk of window columns); 128 rows per block.
template <int M, bool CPLX>
__global__ void __launch_bounds__(128) row_tree3_kernel(const __grid_constant__ Row3Params p) {
    using Tree = SlidingTree3<M>;
    constexpr int n = Tree::kN;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= p.rows) return;
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.P1) return;
    const int qb = min(qa + p.chunk, p.P1);
    const int steps = (qb - qa) + (n - 1);
    const char *xrow = reinterpret_cast<const char *>(p.x) +
                       (p.r_base + row) * p.ld * (int64_t)(CPLX ? sizeof(float2) : sizeof(float));
    float2 *dst = p.z + (int64_t)row * p.zrow + (int64_t)qa * n;
    Tree tree;
    tree.init();
    for (int jb = 0; jb < steps; jb += Tree::kPeriod) {
        static_for<0, Tree::kPeriod>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = qa + j;  // window end column
                const float2 xp = load_x3<CPLX>(xrow, p1);
                const float2 x1 = M >= 1 ? load_x3<CPLX>(xrow, max(p1 - Tree::kS1, 0)) : xp;
                const float2 x2 = M >= 1 ? load_x3<CPLX>(xrow, max(p1 - 2 * Tree::kS1, 0)) : xp;
                float2 o[n];
                tree.template step<J>(p.om, xp, x1, x2, o);
                if (j >= n - 1) {
#pragma unroll
                    for (int k = 0; k < n; ++k) dst[k] = o[k];
                    dst += n;
                }
            }
        });
    }
}

// Column levels: thread = one channel (q1, k1) of z (any n1), 128 channels per block; the
// tile's z rows reach a shared-memory ring one group ahead (cp.async), the level-0
// look-backs 2 s_1 rows up are read from the same ring.
__host__ __device__ constexpr int col3_group(int M) { return M >= 3 ? 6 : 8; }  // multiple of the period
__host__ __device__ constexpr int col3_ring_rows(int M) {
    const int need = (M >= 1 ? 2 * pow3(M - 1) : 0) + 2 * col3_group(M);
    int r = 1;
    while (r < need) r <<= 1;
    return r;
}

__device__ __forceinline__ void cp_async3_8(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}

template <int M>
__global__ void __launch_bounds__(128) col_tree3_kernel(const __grid_constant__ Col3Params p) {
    using Tree = SlidingTree3<M>;
    constexpr int n = Tree::kN;
    constexpr int G = col3_group(M);
    constexpr int RD = col3_ring_rows(M);
    constexpr int S1 = Tree::kS1;
    extern __shared__ float2 ring[];  // RD x 128
    const int CH = blockDim.x;
    const int64_t ch0 = (int64_t)blockIdx.x * CH;
    const int64_t ch = ch0 + threadIdx.x;
    const bool active = ch < p.nch;
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.rows_out) return;  // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const int steps = (qb - qa) + (n - 1);
    const int zr_end = qb + n - 1;  // one past the last z row used

    const int64_t chc = active ? ch : 0;
    const int64_t q1 = chc / p.n1;
    const int64_t k1 = chc - q1 * p.n1;
    float2 *dst = p.out + (int64_t)qa * p.orow + q1 * ((int64_t)n * p.n1) + k1;
    const float s = p.scale;

    auto fetch = [&](int r_lo, int r_hi) {
        for (int rr = r_lo; rr < r_hi; ++rr) {
            const bool ok = ch < p.nch;
            cp_async3_8(&ring[(rr & (RD - 1)) * CH + threadIdx.x], p.z + (int64_t)rr * p.nch + (ok ? ch : 0), ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    Tree tree;
    tree.init();
    fetch(qa - 2 * S1, min(qa + G, zr_end));
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    constexpr int UNR = G;  // a multiple of the tree's period
    for (int jb = 0; jb < steps; jb += UNR) {
        if (jb + UNR < steps) fetch(qa + jb + UNR, min(qa + jb + 2 * UNR, zr_end));
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int zr = qa + j;  // z row = window end row
                const float2 xp = ring[(zr & (RD - 1)) * CH + threadIdx.x];
                const float2 x1 = M >= 1 ? ring[((zr - S1) & (RD - 1)) * CH + threadIdx.x] : xp;
                const float2 x2 = M >= 1 ? ring[((zr - 2 * S1) & (RD - 1)) * CH + threadIdx.x] : xp;
                float2 o[n];
                tree.template step<J % Tree::kPeriod>(p.om, xp, x1, x2, o);
                if (j >= n - 1 && active) {
#pragma unroll
                    for (int k = 0; k < n; ++k) __stcs(dst + (int64_t)k * p.n1, c_scale(s, o[k]));
                    dst += p.orow;
                }
            }
        });
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
    }
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
    dim3 grid((unsigned)((a.rows + 127) / 128), (unsigned)((a.P1 + p.chunk - 1) / p.chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    switch (a.m1 * 2 + (a.cplx ? 1 : 0)) {
        case 0: row_tree3_kernel<0, false><<<grid, 128, 0, s>>>(p); break;
        case 1: row_tree3_kernel<0, true><<<grid, 128, 0, s>>>(p); break;
        case 2: row_tree3_kernel<1, false><<<grid, 128, 0, s>>>(p); break;
        case 3: row_tree3_kernel<1, true><<<grid, 128, 0, s>>>(p); break;
        case 4: row_tree3_kernel<2, false><<<grid, 128, 0, s>>>(p); break;
        case 5: row_tree3_kernel<2, true><<<grid, 128, 0, s>>>(p); break;
        case 6: row_tree3_kernel<3, false><<<grid, 128, 0, s>>>(p); break;
        case 7: row_tree3_kernel<3, true><<<grid, 128, 0, s>>>(p); break;
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
    dim3 grid((unsigned)((nch + 127) / 128), (unsigned)((a.rows_out + p.chunk - 1) / p.chunk));
    if (grid.y > 65535 || grid.x == 0) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * 128 * (size_t)col3_ring_rows(a.m0);
    switch (a.m0) {
        case 0: col_tree3_kernel<0><<<grid, 128, smem, s>>>(p); break;
        case 1: col_tree3_kernel<1><<<grid, 128, smem, s>>>(p); break;
        case 2: col_tree3_kernel<2><<<grid, 128, smem, s>>>(p); break;
        case 3: col_tree3_kernel<3><<<grid, 128, smem, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
