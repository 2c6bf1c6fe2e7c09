// Adjoint passes (transposed tree): launchers.  Instantiations live in adj_m*.cu.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "adjoint_kernels.cuh"
#include "tree_kernels.cuh"

namespace swdft {

// gz[qb + o][ch] += side[b - 1][o][ch] for every chunk boundary qb = b * chunk (b >= 1) and
// o < n0 - 1: the rows two adj_col chunks share.  Grid y = boundary b - 1, z = array; each
// boundary's rows are one contiguous run in gz and in side, added two values (16 bytes) at a
// time when both runs allow it (pairs), else one.
__global__ void __launch_bounds__(256) adj_fold_kernel(const __grid_constant__ AdjFoldParams p) {
    const int64_t b = (int64_t)blockIdx.y + 1;
    float2 *dst = p.gz[blockIdx.z] + b * p.chunk * p.nch;
    const float2 *src = p.side[blockIdx.z] + (b - 1) * p.per_row;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (p.pairs) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.per_row / 2; i += stride) {
            const float4 a = d4[i], v = s4[i];
            d4[i] = make_float4(a.x + v.x, a.y + v.y, a.z + v.z, a.w + v.w);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.per_row; i += stride)
            dst[i] = c_add(dst[i], src[i]);
    }
}

// The column adjoint's staging layout for each (n0, n1) = (2^m0, 2^m1), chosen once.
AdjColLayout adj_col_layout_cached(int m0, int m1) {
    static std::once_flag once;
    static AdjColLayout table[kMaxLog2 + 1][kMaxLog2 + 1];
    std::call_once(once, [] {
        for (int M = 0; M <= kMaxLog2; ++M)
            for (int m = 0; m <= kMaxLog2; ++m) table[M][m] = adj_col_layout(M, adj_col_B(M), m);
    });
    return table[m0][m1];
}

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

int adj_col_launches(int64_t rows_out, int m0, int64_t requested) {
    return rows_out > 0 && adj_side_elems(rows_out, m0, 1, 0, requested) > 0 ? 2 : 1;
}

cudaError_t launch_adj_col(const AdjColArgs &a, cudaStream_t s) {
    const int64_t nch = a.P1 << a.m1;
    const int64_t zrows = a.rows_out + (int64_t(1) << a.m0) - 1;
    if (a.rows_out <= 0 || nch <= 0) return cudaSuccess;
    if (a.m0 < 0 || a.m0 > kMaxLog2 || a.m1 < 0 || a.m1 > kMaxLog2 || zrows > INT32_MAX)
        return cudaErrorInvalidValue;
    if (a.nz < 1 || a.nz > kAdjZ) return cudaErrorInvalidValue;
    AdjColRingParams p;
    for (int z = 0; z < kAdjZ; ++z) {
        p.G[z] = a.G[z];
        p.gz[z] = a.gz[z];
        p.side[z] = a.side[z];
    }
    p.nch = nch;
    p.rows_out = (int)a.rows_out;
    p.chunk = (int)adj_col_chunk(a.rows_out, a.m0, a.chunk);
    const int64_t side_elems = adj_side_elems(a.rows_out, a.m0, a.P1, a.m1, a.chunk);
    for (int z = 0; z < a.nz; ++z)
        if (!a.G[z] || !a.gz[z] || (side_elems > 0 && a.side[z] == nullptr)) return cudaErrorInvalidValue;
    // 8-byte copies need complex64 alignment; 16-byte copies (channel pairs) need n1 >= 2 and
    // G 16-byte aligned (every pair then starts on an even value in G and in the ring)
    for (int z = 0; z < a.nz; ++z)
        if ((uintptr_t)a.G[z] % 8 != 0) return cudaErrorInvalidValue;
    bool q16 = a.m1 >= 1;
    for (int z = 0; z < a.nz; ++z) q16 = q16 && (uintptr_t)a.G[z] % 16 == 0;
    p.q16 = q16 ? 1 : 0;
    p.m1 = a.m1;
    p.scale = a.scale;
    p.L = adj_col_layout_cached(a.m0, a.m1);
    for (int j = 0; j < kMaxN; ++j) p.om64[j] = a.om64[j];
    const int B = adj_col_B(a.m0);  // the one split built per window side
    const int threads = 128;
    const int64_t per_block = threads >> B;
    dim3 grid((unsigned)((nch + per_block - 1) / per_block), (unsigned)((a.rows_out + p.chunk - 1) / p.chunk),
              (unsigned)a.nz);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    const size_t smem = adj_col_smem(a.m0, p.L.slot);
    switch (a.m0) {
#define F(M_)                                                                       \
    case M_:                                                                        \
        adj_col_ring_launch_mb<M_, adj_col_B(M_)>(p, grid, dim3(threads), smem, s); \
        break;
        F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || side_elems == 0) return e;
    // the rows two chunks share: gz += side, one launch for every array
    AdjFoldParams f;
    for (int z = 0; z < kAdjZ; ++z) {
        f.gz[z] = a.gz[z];
        f.side[z] = a.side[z];
    }
    f.nch = nch;
    f.per_row = ((int64_t(1) << a.m0) - 1) * nch;
    f.total = side_elems;
    f.chunk = p.chunk;
    // 16-byte pieces: gz and side 16-byte aligned, and every boundary's run (per_row values,
    // starting chunk * nch values into gz) of an even length at an even offset
    f.pairs = nch % 2 == 0 ? 1 : 0;
    for (int z = 0; z < a.nz; ++z)
        if ((uintptr_t)a.gz[z] % 16 != 0 || (uintptr_t)a.side[z] % 16 != 0) f.pairs = 0;
    const int64_t nb = side_elems / f.per_row;  // chunk boundaries
    if (nb > 65535) return cudaErrorInvalidValue;
    const int64_t pieces = f.pairs ? f.per_row / 2 : f.per_row;
    const int64_t fb = std::max<int64_t>(1, std::min<int64_t>((pieces + 255) / 256, 1024));
    adj_fold_kernel<<<dim3((unsigned)fb, (unsigned)nb, (unsigned)a.nz), 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_adj_row(const AdjRowArgs &a, cudaStream_t s) {
    if (a.zrows <= 0 || a.N1 <= 0) return cudaSuccess;
    if (a.m1 < 0 || a.m1 > kMaxLog2 || a.zrows > INT32_MAX || a.N1 > INT32_MAX) return cudaErrorInvalidValue;
    if (a.nz < 1 || a.nz > kAdjZ) return cudaErrorInvalidValue;
    AdjRowParams p;
    for (int z = 0; z < kAdjZ; ++z) {
        p.gz[z] = a.gz[z];
        p.gx[z] = a.gx[z];
    }
    for (int z = 0; z < a.nz; ++z)
        if (!a.gz[z] || !a.gx[z]) return cudaErrorInvalidValue;
    // 16-byte staging copies of gz rows (n1 >= 2)
    for (int z = 0; z < a.nz; ++z)
        if (a.m1 >= 1 && (uintptr_t)a.gz[z] % 16 != 0) return cudaErrorInvalidValue;
    p.ld_out = a.ld_out;
    p.zrows = (int)a.zrows;
    p.N1 = (int)a.N1;
    p.P1 = (int)(a.N1 - (int64_t(1) << a.m1) + 1);
    for (int j = 0; j < kMaxN; ++j) p.om64[j] = a.om64[j];
    const int B = adj_row_B(a.m1);  // the one split built per window side
    const int threads = 128;
    const int64_t per_block = threads >> B;
    const int64_t row_blocks = (a.zrows + per_block - 1) / per_block;
    int64_t chunk = a.chunk;
    if (chunk <= 0) {
        // as many column chunks as keep one wave of resident blocks busy (the pass is
        // latency-bound: a second, partial wave would nearly double its time), none shorter
        // than n1 (each re-walks n1 - 1 columns of warm-up)
        static std::atomic<int> bps_cache[kMaxLog2 + 1][2];  // 0: not queried yet
        int bps = bps_cache[a.m1][a.cplx ? 1 : 0].load(std::memory_order_relaxed);
        if (bps <= 0) {
            switch (a.m1) {
#define F(M_)                                                  \
    case M_:                                                   \
        bps = adj_row_bps_mb<M_, adj_row_B(M_)>(a.cplx);       \
        break;
                F(0) F(1) F(2) F(3) F(4) F(5) F(6)
#undef F
                default:
                    return cudaErrorInvalidValue;
            }
            bps_cache[a.m1][a.cplx ? 1 : 0].store(bps, std::memory_order_relaxed);
        }
        const int64_t slots = (int64_t)std::max(1, a.sm_count) * std::max(1, bps);
        const int64_t nchunk = std::max<int64_t>(1, slots / std::max<int64_t>(1, row_blocks * a.nz));
        chunk = std::max<int64_t>((a.N1 + nchunk - 1) / nchunk, int64_t(1) << a.m1);
    }
    p.chunk = (int)std::min<int64_t>(chunk, a.N1);
    dim3 grid((unsigned)row_blocks, (unsigned)((a.N1 + p.chunk - 1) / p.chunk), (unsigned)a.nz);
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
