// Column-level pass (Eq. colfswft2d): launcher.  Kernel instantiations live in
// tree_col_m*.cu so they compile in parallel.
#include <algorithm>

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
