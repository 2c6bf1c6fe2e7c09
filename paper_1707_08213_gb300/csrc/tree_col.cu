// Column-level pass (Eq. colfswft2d): launcher.  Kernel instantiations live in
// tree_col_m*.cu so they compile in parallel.
#include <algorithm>
#include <cstring>

#include "tree_kernels.cuh"

namespace swdft {

int col_tree_clamp_B(int m0, int B) { return clamp_split(m0, B); }

int col_tree_clamp_groups(int m0, int B, int groups) {
    // at most 256 threads and a ring within the default 48 KB of dynamic shared memory
    groups = std::max(1, groups);
    while (groups > 1 && (32 * (1 << B) * groups > 256 ||
                          sizeof(float2) * col_ring_rows(m0) * 32 * groups > 48 * 1024))
        groups >>= 1;
    return groups;
}

int col_tree_blocks_per_sm(int m0, int B, int groups) {
    B = col_tree_clamp_B(m0, B);
    groups = col_tree_clamp_groups(m0, B, groups);
    const int threads = 32 * (1 << B) * groups;
    switch (m0 * 8 + B) {
#define F(M_, B_)      \
    case M_ * 8 + B_:  \
        return col_blocks_per_sm<M_, B_>(threads, groups);
        SWDFT_MB_CASES(F)
#undef F
        default:
            return 0;
    }
}

cudaError_t col_tma_status(int *status, bool reset) {
    *status = 0;
    for (int M = 0; M <= kMaxLog2; ++M) {
        int st = 0;
        cudaError_t e = cudaSuccess;
        switch (M) {
#define F(M_)                                  \
    case M_:                                   \
        e = col_tma_status_mb<M_>(&st, reset); \
        break;
            F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
        }
        if (e != cudaSuccess) return e;
        if (st) *status = 1;
    }
    return cudaSuccess;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tiled_encoder() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        return cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                           cudaSuccess &&
                       q == cudaDriverEntryPointSuccess
                   ? reinterpret_cast<EncodeTiledFn>(p)
                   : nullptr;
    }();
    return fn;
}

}  // namespace

cudaError_t launch_col_tree(const ColTreeArgs &a, cudaStream_t s) {
    if (a.P1 < 0 || a.m1 < 0 || a.m1 > kMaxInnerLog2 || a.P1 > (INT64_MAX >> kMaxInnerLog2)) return cudaErrorInvalidValue;
    const int64_t nch = a.P1 << a.m1;
    if (a.rows_out <= 0 || nch <= 0 || a.slices <= 0) return cudaSuccess;
    if (a.m0 < 0 || a.m0 > kMaxLog2 || a.rows_out > INT32_MAX) return cudaErrorInvalidValue;
    ColParams p;
    p.g.z = a.z;
    p.g.out = a.out;
    p.g.nch = nch;
    p.g.orow = nch << a.m0;
    p.g.rows_out = (int)a.rows_out;
    p.g.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.rows_out, a.rows_out);
    p.g.m1 = a.m1;
    p.g.scale = a.scale;
    p.g.zslice = a.z_slice;
    p.g.oslice = a.out_slice;
    const int B = col_tree_clamp_B(a.m0, a.B);
    const int groups = col_tree_clamp_groups(a.m0, B, a.groups);
    p.g.groups = groups;
    for (int j = 0; j < kMaxN; ++j) p.om.w[j] = a.om64[j];
    const int64_t per_block = 32LL * groups;
    const int64_t gx = (nch + per_block - 1) / per_block;
    const int64_t gy = (a.rows_out + p.g.chunk - 1) / p.g.chunk;
    if (gy > 65535 || gx > INT32_MAX) return cudaErrorInvalidValue;
    dim3 block(32 * (1 << B) * groups);
    // one stack of z rows given from its first padding row: the tile's z rows come by TMA
    // (rows 16-byte aligned: nch even, the base aligned; every tile's first channel is even)
    // (its ring holds one more step group: tiles whose ring would pass the default 48 KB of
    // dynamic shared memory keep the cp.async stage)
    const size_t tma_smem = 128 + sizeof(float2) * col_ring_rows(a.m0 < 0 ? 0 : a.m0, kColTmaAhead) * per_block;
    // (chunks must start on whole step groups)
    if (a.z_full && a.slices == 1 && nch % 2 == 0 && (uintptr_t)a.z_full % 16 == 0 && a.z_pad >= 0 &&
        nch <= (int64_t(1) << 32) && a.z == a.z_full + a.z_pad * nch && tma_smem <= 48 * 1024 &&
        p.g.chunk % col_group(a.m0 < 0 ? 0 : a.m0) == 0) {
        EncodeTiledFn enc = tiled_encoder();
        if (enc) {
            ColTmaParams q;
            std::memset(&q, 0, sizeof(q));
            const int64_t rows = a.z_pad + a.rows_out + (int64_t(1) << a.m0) - 1;
            cuuint64_t dims[2] = {(cuuint64_t)nch, (cuuint64_t)rows};
            cuuint64_t strides[1] = {(cuuint64_t)nch * sizeof(float2)};
            cuuint32_t box[2] = {(cuuint32_t)per_block, (cuuint32_t)col_group(a.m0)};
            cuuint32_t estr[2] = {1, 1};
            if (enc(&q.zmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2 *>(a.z_full), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                q.g = p.g;
                q.pad = (int)a.z_pad;
                q.om = p.om;
                dim3 grid((unsigned)gx, (unsigned)gy, 1);
                switch (a.m0 * 8 + B) {
#define F(M_, B_)                                      \
    case M_ * 8 + B_:                                  \
        col_tma_launch_mb<M_, B_>(q, grid, block, s);  \
        break;
                    SWDFT_MB_CASES(F)
#undef F
                    default:
                        return cudaErrorInvalidValue;
                }
                return cudaGetLastError();
            }
        }
    }
    // slices beyond the grid's z limit go out as further launches with shifted bases
    constexpr int64_t kMaxZ = 65535;
    for (int64_t s0 = 0; s0 < a.slices; s0 += kMaxZ) {
        const int64_t ns = std::min(kMaxZ, a.slices - s0);
        p.g.z = a.z + s0 * a.z_slice;
        p.g.out = a.out + s0 * a.out_slice;
        dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)ns);
        switch (a.m0 * 8 + B) {
#define F(M_, B_)                                  \
    case M_ * 8 + B_:                              \
        col_launch_mb<M_, B_>(p, grid, block, s);  \
        break;
            SWDFT_MB_CASES(F)
#undef F
            default:
                return cudaErrorInvalidValue;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int fused_col_B(int m0) { return m0 >= 6 ? 3 : std::min(m0, 2); }

cudaError_t launch_fused_tree(const FusedTreeArgs &a, cudaStream_t s) {
    const int64_t nch = a.P1 << a.m1;
    if (a.rows_out <= 0 || nch <= 0) return cudaSuccess;
    if (a.m0 < 0 || a.m0 > kMaxLog2 || !fused_supported(a.m0, a.m1) || a.rows_out > INT32_MAX || a.P1 > INT32_MAX)
        return cudaErrorInvalidValue;
    FusedParams p;
    p.g.z = nullptr;
    p.g.out = a.out;
    p.g.nch = nch;
    p.g.orow = nch << a.m0;
    p.g.rows_out = (int)a.rows_out;
    p.g.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.rows_out, a.rows_out);
    p.g.m1 = a.m1;
    p.g.scale = a.scale;
    p.g.zslice = 0;
    p.g.oslice = 0;
    const int B = fused_col_B(a.m0);
    // n1 = 64: a tile holds whole window columns (an even number of 32-channel groups)
    p.g.groups = a.m1 == 6 ? std::max(2, col_tree_clamp_groups(a.m0, B, a.groups) & ~1)
                           : col_tree_clamp_groups(a.m0, B, a.groups);
    p.x = a.x;
    p.ld = a.ld;
    p.zrows = (int)(a.rows_out + (int64_t(1) << a.m0) - 1);
    p.P1 = (int)a.P1;
    for (int j = 0; j < kMaxN; ++j) p.om.w[j] = a.om64[j];
    const int64_t per_block = 32LL * p.g.groups;
    dim3 grid((unsigned)((nch + per_block - 1) / per_block), (unsigned)((a.rows_out + p.g.chunk - 1) / p.g.chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    dim3 block(32 * (1 << B) * p.g.groups);
    switch (a.m0) {
        case 0: fused_launch_mb<0, 0>(p, a.m1, a.cplx, grid, block, s); break;
        case 1: fused_launch_mb<1, 1>(p, a.m1, a.cplx, grid, block, s); break;
        case 2: fused_launch_mb<2, 2>(p, a.m1, a.cplx, grid, block, s); break;
        case 3: fused_launch_mb<3, 2>(p, a.m1, a.cplx, grid, block, s); break;
        case 4: fused_launch_mb<4, 2>(p, a.m1, a.cplx, grid, block, s); break;
        case 5: fused_launch_mb<5, 2>(p, a.m1, a.cplx, grid, block, s); break;
        case 6: fused_launch_mb<6, 3>(p, a.m1, a.cplx, grid, block, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
