// Adjoint passes (transposed tree): launchers.  Instantiations live in adj_m*.cu.
#include <algorithm>

#include "adjoint_kernels.cuh"
#include "tree_kernels.cuh"

namespace swdft {

int64_t adj_col_chunk(int64_t rows_out, int m0, int64_t requested) {
    const int64_t n = int64_t(1) << m0;
    int64_t chunk = requested > 0 ? requested : rows_out;
    chunk = std::max<int64_t>(chunk, n - 1);  // a z row is shared by at most two chunks
    return std::max<int64_t>(1, std::min(chunk, rows_out));
}

int64_t adj_side_elems(int64_t rows_out, int m0, int64_t P1, int m1, int64_t requested) {
    if (rows_out <= 0) return 0;
    const int64_t chunk = adj_col_chunk(rows_out, m0, requested);
    const int64_t nchunks = (rows_out + chunk - 1) / chunk;
    return (nchunks - 1) * ((int64_t(1) << m0) - 1) * (P1 << m1);
}

int adj_row_split(int m1) { return adj_row_B(m1); }

cudaError_t launch_adj_col(const AdjColArgs &a, cudaStream_t s) {
    const int64_t nch = a.P1 << a.m1;
    const int64_t zrows = a.rows_out + (int64_t(1) << a.m0) - 1;
    if (a.rows_out <= 0 || nch <= 0) return cudaSuccess;
    if (a.m0 < 0 || a.m0 > kMaxLog2 || a.m1 < 0 || a.m1 > kMaxLog2 || zrows > INT32_MAX)
        return cudaErrorInvalidValue;
    if (a.nz < 1 || a.nz > kAdjZ) return cudaErrorInvalidValue;
    AdjColParams p;
    for (int z = 0; z < kAdjZ; ++z) {
        p.G[z] = a.G[z];
        p.gz[z] = a.gz[z];
        p.side[z] = a.side[z];
    }
    p.nch = nch;
    p.rows_out = (int)a.rows_out;
    p.chunk = (int)adj_col_chunk(a.rows_out, a.m0, a.chunk);
    for (int z = 0; z < a.nz; ++z)
        if (!a.G[z] || !a.gz[z] || (p.chunk < a.rows_out && a.m0 > 0 && a.side[z] == nullptr))
            return cudaErrorInvalidValue;
    p.m1 = a.m1;
    p.scale = a.scale;
    for (int j = 0; j < kMaxN; ++j) p.om64[j] = a.om64[j];
    const int B = adj_col_B(a.m0);  // the one split built per window side
    const int threads = 128;
    const int64_t per_block = threads >> B;
    dim3 grid((unsigned)((nch + per_block - 1) / per_block), (unsigned)((a.rows_out + p.chunk - 1) / p.chunk),
              (unsigned)a.nz);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    switch (a.m0) {
#define F(M_)                                                                \
    case M_:                                                                 \
        adj_col_launch_mb<M_, adj_col_B(M_)>(p, grid, dim3(threads), s);     \
        break;
        F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_row(const AdjRowArgs &a, cudaStream_t s) {
    if (a.zrows <= 0 || a.N1 <= 0) return cudaSuccess;
    if (a.m1 < 0 || a.m1 > kMaxLog2 || a.zrows > INT32_MAX || a.N1 > INT32_MAX) return cudaErrorInvalidValue;
    if (a.nz < 1 || a.nz > kAdjZ) return cudaErrorInvalidValue;
    AdjRowParams p;
    for (int z = 0; z < kAdjZ; ++z) {
        p.gz[z] = a.gz[z];
        p.side[z] = a.side[z];
        p.gx[z] = a.gx[z];
    }
    for (int z = 0; z < a.nz; ++z)
        if (!a.gz[z] || !a.gx[z]) return cudaErrorInvalidValue;
    if (a.m0 < 0 || a.m0 > kMaxLog2 || a.rows_out > INT32_MAX) return cudaErrorInvalidValue;
    p.col_chunk = (int)adj_col_chunk(a.rows_out, a.m0, a.col_chunk);
    p.rows_out = (int)a.rows_out;
    p.n0m1 = (1 << a.m0) - 1;
    p.ld_out = a.ld_out;
    p.zrows = (int)a.zrows;
    p.N1 = (int)a.N1;
    p.P1 = (int)(a.N1 - (int64_t(1) << a.m1) + 1);
    p.chunk = (int)std::min<int64_t>(a.chunk > 0 ? a.chunk : a.N1, a.N1);
    for (int j = 0; j < kMaxN; ++j) p.om64[j] = a.om64[j];
    const int B = adj_row_B(a.m1);  // the one split built per window side
    const int threads = 128;
    const int64_t per_block = threads >> B;
    dim3 grid((unsigned)((a.zrows + per_block - 1) / per_block), (unsigned)((a.N1 + p.chunk - 1) / p.chunk),
              (unsigned)a.nz);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    switch (a.m1) {
#define F(M_)                                                                         \
    case M_:                                                                          \
        adj_row_launch_mb<M_, adj_row_B(M_)>(p, a.cplx, grid, dim3(threads), s);      \
        break;
        F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
