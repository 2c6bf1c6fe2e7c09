// Ternary and mixed-radix tree passes (windows of 3^b 2^a samples, b >= 1, at most 64, along
// an axis): launchers.  Kernels in tree3_kernels.cuh, instantiated in tree3_row.cu and
// tree3_col.cu.
#include <algorithm>

#include "tree3_kernels.cuh"

namespace swdft {

// w_n^{-j} for the axis's window length (FP64-evaluated, FP32-rounded) and h = sin(pi/3)
// = -Im w_n^{-n/3} (n a multiple of 3; unused for n = 1).
static void fill_omega_n(OmegaN &om, int n) {
    make_omega(n, om.w);
    for (int j = n; j < kMaxN; ++j) om.w[j] = make_float2(0.f, 0.f);
    om.h = n % 3 == 0 ? -om.w[n / 3].y : 0.f;
}

static bool mixed_built(int b, int a) {
    return (b == 0 && a == 0) || (b >= 1 && b <= kMaxLog3 && a >= 0 && mixed_n(b, a) <= kMaxN);
}

cudaError_t launch_row_tree3(const Row3Args &a, cudaStream_t s) {
    if (a.rows <= 0 || a.P1 <= 0) return cudaSuccess;
    if (!mixed_built(a.b1, a.a1) || a.rows > INT32_MAX || a.P1 > INT32_MAX) return cudaErrorInvalidValue;
    const int n1 = mixed_n(a.b1, a.a1);
    Row3Params p;
    p.x = a.x;
    p.ld = a.ld;
    p.r_base = a.r_base;
    p.zrow = a.P1 * n1;
    p.rows = (int)a.rows;
    p.P1 = (int)a.P1;
    p.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.P1, a.P1);
    p.z = a.z;
    fill_omega_n(p.om, n1);
    dim3 grid((unsigned)((a.rows + 31) / 32), (unsigned)((a.P1 + p.chunk - 1) / p.chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    const dim3 block(a.b1 >= 1 ? 96 : 32);  // a warp per residue of the split tree
    switch (a.b1 * 8 + a.a1) {
#define F(B3_, A2_)                                               \
    case B3_ * 8 + A2_:                                           \
        row3_launch_ba<B3_, A2_>(p, a.cplx ? 1 : 0, grid, block, s); \
        break;
        SWDFT_MIXED_CASES(F)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_col_tree3(const Col3Args &a, cudaStream_t s) {
    if (a.n1 < 1 || a.P1 < 0) return cudaErrorInvalidValue;
    const int64_t nch = a.P1 * a.n1;
    if (a.rows_out <= 0 || nch <= 0) return cudaSuccess;
    if (!mixed_built(a.b0, a.a0) || a.rows_out > INT32_MAX) return cudaErrorInvalidValue;
    const int n0 = mixed_n(a.b0, a.a0);
    Col3Params p;
    p.z = a.z;
    p.out = a.out;
    p.nch = nch;
    p.orow = nch * n0;
    p.rows_out = (int)a.rows_out;
    p.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.rows_out, a.rows_out);
    p.n1 = a.n1;
    p.scale = a.scale;
    fill_omega_n(p.om, n0);
    if (a.n1 > kCol3Ch) return cudaErrorInvalidValue;
    const int64_t T = std::max(1, kCol3Ch / a.n1);  // whole window columns per tile
    dim3 grid((unsigned)((a.P1 + T - 1) / T), (unsigned)((a.rows_out + p.chunk - 1) / p.chunk));
    if (grid.y > 65535 || grid.x == 0) return cudaErrorInvalidValue;
    const dim3 block(a.b0 >= 1 ? 3 * kCol3Ch : kCol3Ch);  // a warp per (residue, 32 channels)
    const int staged = a.n1 % 4 != 0 ? 1 : 0;
    switch (a.b0 * 8 + a.a0) {
#define F(B3_, A2_)                                          \
    case B3_ * 8 + A2_:                                      \
        col3_launch_ba<B3_, A2_>(p, staged, grid, block, s); \
        break;
        SWDFT_MIXED_CASES(F)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
