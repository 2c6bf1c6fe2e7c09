// Adjoint for ternary and mixed-radix windows (n = 3^b 2^a along an axis, b >= 1): the
// overlap-add of every window's inverse DFT (the transpose of Eq. 2's map), evaluated per axis
// in gather form with an inverse FFT of length n per window:
//
//   column pass  gz[r][q1][k1] = c sum_{q0 = r-n0+1..r} sum_k0 G[q0][q1][k0][k1] w_{n0}^{+(r-q0) k0}
//   row pass     gx[r][p1]     =   sum_{q1 = p1-n1+1..p1} sum_k1 gz[r][q1][k1] w_{n1}^{+(p1-q1) k1}
//
// (only windows that exist contribute; gx keeps the real part for real input).  A thread walks
// its channel (column pass) or its row (row pass) window by window: it computes the window's
// n inverse-DFT values from the n spectral values it loads (an in-place mixed-radix inverse
// FFT in registers, radix 3 and 2 steps, every index fixed at compile time; twiddles from the
// kernel parameters) and adds value j into a ring of n partial
// outputs in shared memory, one slot per output row (column) still open; after window q the
// output at q has all its windows and leaves the ring.  Chunks of windows run in parallel:
// the n - 1 outputs a chunk shares with each neighbour are added atomically into a zeroed
// buffer, the others stored.  An axis whose window is a power of two uses the transposed
// radix-2 tree instead (adj_row_kernel).
#include <algorithm>

#include "tree3_core.cuh"

namespace swdft {

struct Adj3ColParams {
    const float2 *G;  // [rows_out][P1][n0][n1]
    float2 *gz;       // [rows_out + n0 - 1][P1][n1], zeroed before the launch
    int64_t nch;      // P1 * n1
    int n1;
    int rows_out;
    int chunk;        // windows per thread
    float scale;
    OmegaN om;        // w_{n0}^{-j}
};

struct Adj3RowParams {
    const float2 *gz;  // [zrows][P1][n1]
    void *gx;          // [zrows][ld_out] float or float2, zeroed before the launch
    int64_t ld_out;
    int zrows, N1, P1;
    int chunk;         // windows (columns q1) per thread
    int row_blocks;    // blocks along the rows (grid x)
    OmegaN om;         // w_{n1}^{-j}
};

constexpr int kAdj3Threads = 128;
constexpr int64_t kAdj3Blocks = 152 * 8;  // blocks a pass is cut into (about eight per SM)

__device__ __forceinline__ float2 conj_mul(float2 w, float2 v) {  // conj(w) v
    return make_float2(w.x * v.x + w.y * v.y, w.x * v.y - w.y * v.x);
}

__device__ __forceinline__ void atomic_add2(float2 *d, float2 v) {
    atomicAdd(&d->x, v.x);
    atomicAdd(&d->y, v.y);
}

// The window's inverse DFT, X[j] = sum_k v[k] w_N^{+jk} (unnormalised), in place by
// decimation in time: N = R M (radix R = 3 while N has a factor 3 above 3, then 2), the R
// interleaved subsequences v[d], v[d + R], ... transformed recursively in place, then per
// j' < M one R-point butterfly on their outputs twiddled by w_N^{+j' d} (no twiddle for
// j' = 0), its output a stored back over input d.  Inputs in natural order; X[j] ends at
// position ifft_pos(N, j) = R ifft_pos(M, j mod M) + j / M (digit-reversed), all indices fixed
// at compile time; twiddles w_N^{+x} = conj(w_NTOP^{-x NTOP / N}) from the kernel parameters'
// table for the top length NTOP.  The 2-point butterfly is a sum and a difference; the
// 3-point one, with s = t1 + t2, d = t1 - t2 and m = t0 - s/2, is X0 = t0 + s,
// X1 = m + i h d, X2 = m - i h d (w_3^{+1} = -1/2 + i h, h = sin(pi/3)), each component of
// X1 and X2 one fused multiply-add.
__host__ __device__ constexpr int ifft_radix(int n) { return (n % 3 == 0 && n > 3) ? 3 : ((n % 2 == 0 && n > 2) ? 2 : n); }
__host__ __device__ constexpr int ifft_pos(int n, int j) {
    return n <= 3 ? j : ifft_radix(n) * ifft_pos(n / ifft_radix(n), j % (n / ifft_radix(n))) + j / (n / ifft_radix(n));
}

__device__ __forceinline__ void ibfly3(float2 t0, float2 t1, float2 t2, float h, float2 &x0, float2 &x1, float2 &x2) {
    const float2 s = c_add(t1, t2);
    const float2 d = c_sub(t1, t2);
    const float2 m = make_float2(fmaf(-0.5f, s.x, t0.x), fmaf(-0.5f, s.y, t0.y));
    x0 = c_add(t0, s);
    x1 = make_float2(fmaf(-h, d.y, m.x), fmaf(h, d.x, m.y));
    x2 = make_float2(fmaf(h, d.y, m.x), fmaf(-h, d.x, m.y));
}

template <int NTOP, int N, int STRIDE, int OFF, int NV>
__device__ __forceinline__ void ifft_rec(float2 (&v)[NV], const OmegaN &om) {
    if constexpr (N == 2) {
        const float2 a = v[OFF], b = v[OFF + STRIDE];
        v[OFF] = c_add(a, b);
        v[OFF + STRIDE] = c_sub(a, b);
    } else if constexpr (N == 3) {
        ibfly3(v[OFF], v[OFF + STRIDE], v[OFF + 2 * STRIDE], om.h, v[OFF], v[OFF + STRIDE], v[OFF + 2 * STRIDE]);
    } else if constexpr (N > 3) {
        constexpr int R = ifft_radix(N), M = N / R;
        static_for<0, R>([&](auto DD) {
            constexpr int d = decltype(DD)::value;
            ifft_rec<NTOP, M, STRIDE * R, OFF + STRIDE * d>(v, om);
        });
        static_for<0, M>([&](auto JJ) {
            constexpr int jp = decltype(JJ)::value;
            constexpr int base = OFF + STRIDE * R * ifft_pos(M, jp);
            float2 t[R];
            static_for<0, R>([&](auto DD) {
                constexpr int d = decltype(DD)::value;
                if constexpr (d == 0 || jp == 0)
                    t[d] = v[base + STRIDE * d];
                else
                    t[d] = conj_mul(om.w[(jp * d * (NTOP / N)) % NTOP], v[base + STRIDE * d]);
            });
            if constexpr (R == 3) {
                ibfly3(t[0], t[1], t[2], om.h, v[base], v[base + STRIDE], v[base + 2 * STRIDE]);
            } else {
                v[base] = c_add(t[0], t[1]);
                v[base + STRIDE] = c_sub(t[0], t[1]);
            }
        });
    }
}

// The window's inverse DFT values, value j added into ring slot slot + j (mod N).
template <int N>
__device__ __forceinline__ void idft_into_ring(float2 (&v)[N], const OmegaN &om, float2 *ring, int slot) {
    ifft_rec<N, N, 1, 0>(v, om);
    static_for<0, N>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        const float2 h = v[ifft_pos(N, j)];
        int sj = slot + j;
        if (sj >= N) sj -= N;
        float2 *a = ring + sj * kAdj3Threads;
        a->x += h.x;
        a->y += h.y;
    });
}

template <int N0>
__global__ void __launch_bounds__(kAdj3Threads) adj3_col_kernel(const __grid_constant__ Adj3ColParams p) {
    extern __shared__ float2 adj3_ring[];  // [N0][kAdj3Threads]
    const int t = threadIdx.x;
    float2 *ring = adj3_ring + t;
    const int64_t ch = (int64_t)blockIdx.x * kAdj3Threads + t;
    const bool active = ch < p.nch;
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.rows_out) return;  // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const int64_t q1 = active ? ch / p.n1 : 0, k1 = active ? ch - q1 * p.n1 : 0;
    const float2 *g = p.G + q1 * (int64_t)N0 * p.n1 + k1;
    const int64_t grow = p.nch * N0;  // elements of G per window row
    float2 *dst = p.gz + ch;
#pragma unroll
    for (int j = 0; j < N0; ++j) ring[j * kAdj3Threads] = make_float2(0.f, 0.f);
    int slot = 0;  // ring slot of output row q0: (q0 - qa) mod N0
    for (int q0 = qa; q0 < qb; ++q0) {
        float2 v[N0];
#pragma unroll
        for (int k0 = 0; k0 < N0; ++k0)
            v[k0] = active ? __ldg(g + (int64_t)q0 * grow + (int64_t)k0 * p.n1) : make_float2(0.f, 0.f);
        idft_into_ring<N0>(v, p.om, ring, slot);
        // row q0 has all its windows (q0 - N0 + 1 .. q0) from this chunk
        float2 *a = ring + slot * kAdj3Threads;
        const float2 o = make_float2(a->x * p.scale, a->y * p.scale);
        *a = make_float2(0.f, 0.f);
        if (active) {
            if (q0 >= qa + N0 - 1)
                dst[(int64_t)q0 * p.nch] = o;  // no other chunk reaches this row
            else
                atomic_add2(dst + (int64_t)q0 * p.nch, o);
        }
        if (++slot == N0) slot = 0;
    }
    // rows qb .. qb + N0 - 2 also take windows of the next chunk
    for (int i = 0; i + 1 < N0; ++i) {
        float2 *a = ring + slot * kAdj3Threads;
        if (active) atomic_add2(dst + (int64_t)(qb + i) * p.nch, make_float2(a->x * p.scale, a->y * p.scale));
        if (++slot == N0) slot = 0;
    }
}

template <int N1, bool CPLX>
__global__ void __launch_bounds__(kAdj3Threads) adj3_row_kernel(const __grid_constant__ Adj3RowParams p) {
    extern __shared__ float2 adj3_ring[];  // [N1][kAdj3Threads]
    const int t = threadIdx.x;
    float2 *ring = adj3_ring + t;
    const int r = blockIdx.x * kAdj3Threads + t;  // z row
    const bool active = r < p.zrows;
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.P1) return;  // uniform per block
    const int qb = min(qa + p.chunk, p.P1);
    const float2 *g = p.gz + (int64_t)(active ? r : 0) * p.P1 * N1;
#pragma unroll
    for (int j = 0; j < N1; ++j) ring[j * kAdj3Threads] = make_float2(0.f, 0.f);
    auto put = [&](int c, float2 o, bool alone) {
        if (!active) return;
        if (CPLX) {
            float2 *d = static_cast<float2 *>(p.gx) + (int64_t)r * p.ld_out + c;
            if (alone)
                *d = o;
            else
                atomic_add2(d, o);
        } else {
            float *d = static_cast<float *>(p.gx) + (int64_t)r * p.ld_out + c;
            if (alone)
                *d = o.x;
            else
                atomicAdd(d, o.x);
        }
    };
    int slot = 0;  // ring slot of output column c: (c - qa) mod N1
    for (int q1 = qa; q1 < qb; ++q1) {
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = active ? __ldg(g + (int64_t)q1 * N1 + k1) : make_float2(0.f, 0.f);
        idft_into_ring<N1>(v, p.om, ring, slot);
        float2 *a = ring + slot * kAdj3Threads;
        put(q1, *a, q1 >= qa + N1 - 1);
        *a = make_float2(0.f, 0.f);
        if (++slot == N1) slot = 0;
    }
    for (int i = 0; i + 1 < N1; ++i) {
        put(qb + i, ring[slot * kAdj3Threads], false);
        if (++slot == N1) slot = 0;
    }
}

// window lengths of the dense passes: 1 and every 3^b 2^a <= 64 with b >= 1
#define SWDFT_ADJ3_CASES(F) F(1) F(3) F(6) F(9) F(12) F(18) F(24) F(27) F(36) F(48) F(54)

// Resident blocks per SM of one instantiation (occupancy API; 1 if the query fails).
template <class K>
static int adj3_bps(K kernel, size_t smem) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, kAdj3Threads, smem) != cudaSuccess || bps < 1)
        bps = 1;
    return bps;
}

// Windows per block along the chunked dimension: `blocks` blocks across it, `units` windows
// along it, `slots` blocks resident at once.  Chunks cost nothing but the atomic adds of
// their n - 1 shared outputs (no warm-up: every window is transformed once), so the count is
// the one that minimises whole waves x windows per block (a last wave that is mostly empty
// leaves most SMs idle), with at least 4 windows per block.
static int adj3_chunk(int64_t units, int64_t blocks, int64_t slots) {
    int64_t best = units, best_cost = INT64_MAX;
    for (int64_t nc = 1; nc <= std::min<int64_t>(units, 256); ++nc) {
        const int64_t chunk = (units + nc - 1) / nc;
        if (chunk < 4 && nc > 1) break;
        const int64_t waves = (blocks * ((units + chunk - 1) / chunk) + slots - 1) / slots;
        const int64_t cost = waves * chunk;
        if (cost < best_cost) {
            best_cost = cost;
            best = chunk;
        }
    }
    return (int)best;
}

static int sm_count_now() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
        sms = 152;
    return sms;
}

static void fill_omega_adj(OmegaN &om, int n) {
    make_omega(n, om.w);
    for (int j = n; j < kMaxN; ++j) om.w[j] = make_float2(0.f, 0.f);
    om.h = n % 3 == 0 ? -om.w[n / 3].y : 0.f;  // sin(pi/3) from the same table
}

cudaError_t launch_adj3_col(const Adj3ColArgs &a, cudaStream_t s) {
    if (a.rows_out <= 0 || a.P1 <= 0) return cudaSuccess;
    if (!a.G || !a.gz || a.n0 < 1 || a.n0 > kMaxN || a.n1 < 1 || a.rows_out > INT32_MAX) return cudaErrorInvalidValue;
    const int64_t nch = a.P1 * a.n1;
    const int64_t zrows = a.rows_out + a.n0 - 1;
    cudaError_t e = cudaMemsetAsync(a.gz, 0, sizeof(float2) * (size_t)(zrows * nch), s);
    if (e != cudaSuccess) return e;
    Adj3ColParams p;
    p.G = a.G;
    p.gz = a.gz;
    p.nch = nch;
    p.n1 = a.n1;
    p.rows_out = (int)a.rows_out;
    const int64_t cblocks = (nch + kAdj3Threads - 1) / kAdj3Threads;
    p.scale = a.scale;
    fill_omega_adj(p.om, a.n0);
    if (cblocks > INT32_MAX) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * (size_t)a.n0 * kAdj3Threads;
    const int64_t sms = sm_count_now();
    switch (a.n0) {
#define F(N_)                                                                                            \
    case N_: {                                                                                           \
        if (smem > 48 * 1024 &&                                                                          \
            (e = cudaFuncSetAttribute(adj3_col_kernel<N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)smem)) != cudaSuccess)                                        \
            return e;                                                                                    \
        static const int bps = adj3_bps(adj3_col_kernel<N_>, smem);                                      \
        p.chunk = adj3_chunk(a.rows_out, cblocks, sms * bps);                                            \
        const dim3 grid((unsigned)cblocks, (unsigned)((a.rows_out + p.chunk - 1) / p.chunk));            \
        if (grid.y > 65535) return cudaErrorInvalidValue;                                                \
        adj3_col_kernel<N_><<<grid, kAdj3Threads, smem, s>>>(p);                                         \
        break;                                                                                           \
    }
        SWDFT_ADJ3_CASES(F)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj3_row(const Adj3RowArgs &a, cudaStream_t s) {
    if (a.zrows <= 0 || a.N1 <= 0) return cudaSuccess;
    if (!a.gz || !a.gx || a.n1 < 1 || a.n1 > a.N1 || a.zrows > INT32_MAX || a.N1 > INT32_MAX)
        return cudaErrorInvalidValue;
    if (a.ld_out != a.N1) return cudaErrorInvalidValue;  // gradient rows are contiguous
    const size_t elem = a.cplx ? sizeof(float2) : sizeof(float);
    cudaError_t e = cudaMemsetAsync(a.gx, 0, (size_t)(a.zrows * a.N1) * elem, s);
    if (e != cudaSuccess) return e;
    Adj3RowParams p;
    p.gz = a.gz;
    p.gx = a.gx;
    p.ld_out = a.ld_out;
    p.zrows = (int)a.zrows;
    p.N1 = (int)a.N1;
    p.P1 = (int)(a.N1 - a.n1 + 1);
    const int64_t rblocks = (a.zrows + kAdj3Threads - 1) / kAdj3Threads;
    const int64_t want = std::max<int64_t>(1, (kAdj3Blocks + rblocks - 1) / rblocks);
    p.chunk = (int)std::min<int64_t>(p.P1, std::max<int64_t>(4, (p.P1 + want - 1) / want));
    p.row_blocks = (int)rblocks;
    fill_omega_adj(p.om, a.n1);
    const dim3 grid((unsigned)rblocks, (unsigned)((p.P1 + p.chunk - 1) / p.chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * (size_t)a.n1 * kAdj3Threads;
    switch (a.n1) {
#define F(N_)                                                                                                \
    case N_:                                                                                                 \
        if (smem > 48 * 1024 &&                                                                              \
            ((e = cudaFuncSetAttribute(adj3_row_kernel<N_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                       (int)smem)) != cudaSuccess ||                                         \
             (e = cudaFuncSetAttribute(adj3_row_kernel<N_, false>,                                           \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)) \
            return e;                                                                                        \
        if (a.cplx)                                                                                          \
            adj3_row_kernel<N_, true><<<grid, kAdj3Threads, smem, s>>>(p);                                   \
        else                                                                                                 \
            adj3_row_kernel<N_, false><<<grid, kAdj3Threads, smem, s>>>(p);                                  \
        break;
        SWDFT_ADJ3_CASES(F)
#undef F
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace swdft
