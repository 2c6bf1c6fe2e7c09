// Dense-contraction form of the 2D sliding window DFT on tcgen05 tensor cores.
//
// The row-column factorisation of Section 4.2 writes every window's 2D DFT as a row DFT
// followed by a column DFT.  Here the column DFT is a matrix product against the n0-point
// DFT matrix F0[j0][k0] = w_{n0}^{-j0 k0}, one product per window row q0 and block of 128
// channels (channel = (q1, k1), the columns of z):
//
//     a[q0][ch][k0] = c * sum_{j0} z[q0 + j0][ch] * F0[j0][k0]
//
// realified as D (128 x 2n0) = A (128 x 2n0) * B (2n0 x 2n0) with A = [Re z | Im z] and
// B = [[C, -S], [S, C]] (C = cos, S = sin of 2 pi j0 k0 / n0).  A is MN-major in shared
// memory: channels are contiguous in z, and the n0 rows a window needs are consecutive
// 16-byte rows of the staged tile, so sliding the window by one row moves the descriptor
// start by 16 bytes -- every window row of the CTA's chunk reuses one TMA-loaded tile.
//
// Precision: operands are bf16 (or fp16) with fp32 accumulation in TMEM.  The 3-term split
// keeps v = hi + lo (hi = bf16(v), lo = bf16(v - hi)) for both z and F0 and accumulates
// hi*hi + hi*lo + lo*hi, dropping only lo*lo (~2^-16 relative per product).
//
// One CTA = 128 channels = the 128 TMEM lanes, with two threads per channel (256 threads).
// Thread 0 issues the TMA loads and the UMMAs; every wait on an mbarrier is bounded and a
// time-out sets an error word and skips ahead to the TMEM release.  The epilogue reads D with
// tcgen05.ld and each thread stores half of its channel's n0 coefficients: for fixed k0 a
// warp writes 32 consecutive channels (256 contiguous bytes), the same pattern as the tree
// kernel.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "sm100_ptx.cuh"
#include "swdft_internal.h"

namespace swdft {

__device__ int g_tc_status;  // 0 = ok; 1 = an mbarrier wait timed out

constexpr int TC_CH = 128;      // channels per CTA = UMMA M = TMEM lanes
constexpr int TCC_THREADS = 256;  // column GEMM: two threads per channel (TMEM lane), k0 halves
constexpr uint32_t TC_MAX_POLLS = 4000;  // x up to ~1 ms per poll

struct TcColParams {
    CUtensorMap planes[4];  // z operand planes: Re hi, Im hi, Re lo, Im lo (2D [rows][nch])
    float2 *out;
    int64_t nch;            // channels = P1 * n1
    int64_t orow;           // output elements per window row
    int rows_out;           // window rows
    int chunk;              // window rows per CTA
    int rz;                 // staged rows per plane (chunk + n0 - 1, rounded up to 8)
    int m1;
    float scale;
    const float *amax;      // per-image fp16 scaling: amax * amax_mult bounds |z| (null: none)
    float amax_mult;
    float2 om64[kMaxN];
};

// Power-of-two scale that brings a bound on the largest |value| of z, amax * mult, to
// [2^13, 2^14): fp16 then keeps its full 11-bit precision without overflow (max 65504).
__device__ __forceinline__ float fp16_prescale(const float *amax, float mult = 1.f) {
    if (!amax) return 1.f;
    const float m = *amax * mult;
    if (!(m > 0.f) || !isfinite(m)) return 1.f;
    int e;
    frexpf(m, &e);              // m = f * 2^e, f in [0.5, 1)
    return ldexpf(1.f, 14 - e);
}

// max |Re|, |Im| over rows x cols of a strided float32 (cplx = 0) or complex64 array
__global__ void __launch_bounds__(256) amax_x_kernel(const void *__restrict__ x, int64_t ld, int64_t rows,
                                                     int64_t cols, int cplx, float *amax) {
    float m = 0.f;
    const int64_t n = rows * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i - (i / cols) * cols;
        if (cplx) {
            const float2 v = reinterpret_cast<const float2 *>(x)[r * ld + c];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        } else {
            m = fmaxf(m, fabsf(reinterpret_cast<const float *>(x)[r * ld + c]));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(amax), __float_as_int(m));
}

template <bool F16>
__device__ __forceinline__ uint16_t to_bits(float v) {
    if constexpr (F16) {
        __half h = __float2half_rn(v);
        return *reinterpret_cast<uint16_t *>(&h);
    } else {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        return *reinterpret_cast<uint16_t *>(&h);
    }
}
template <bool F16>
__device__ __forceinline__ float from_bits(uint16_t b) {
    if constexpr (F16) {
        return __half2float(*reinterpret_cast<__half *>(&b));
    } else {
        return __bfloat162float(*reinterpret_cast<__nv_bfloat16 *>(&b));
    }
}

// Two values as packed 16-bit pairs (first value in the low half): hi = round(v) and
// lo = round(v - hi), with one paired conversion for each (the same bits as converting
// each value on its own).
template <bool F16>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &lo) {
    if constexpr (F16) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Byte offset of element (n, k) in a K-major, no-swizzle operand of K columns: 8x8 core
// matrices of 128 bytes, K-adjacent core matrices 128 B apart, 8-row groups K*16 B apart.
__device__ __forceinline__ uint32_t kmajor_off(int n, int k, int K) {
    return (uint32_t)(((n >> 3) * (K >> 3) + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

template <int M0, int TERMS, bool F16>
__global__ void __launch_bounds__(TCC_THREADS) tc_col_kernel(const __grid_constant__ TcColParams p) {
    constexpr int n0 = 1 << M0;
    constexpr int K = 2 * n0;   // realified contraction length
    constexpr int N = 2 * n0;   // realified output columns (Re k0 | Im k0)
    constexpr int KS = K / 16;  // UMMA k-steps per term
    constexpr int NB = TERMS == 3 ? 2 : 1;       // B tiles (hi, lo)
    constexpr int NP = TERMS == 3 ? 4 : 2;       // A planes
    constexpr uint32_t TMEM_COLS = (2 * N) < 32 ? 32 : 2 * N;  // two accumulator buffers
    constexpr uint32_t B_BYTES = N * K * 2;
    constexpr uint32_t IDESC = umma_idesc_f16(TC_CH, N, !F16, /*a_mn=*/true, /*b_mn=*/false);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base (the launch requests 1 KB of slack)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int rz = p.rz;
    const uint32_t plane_bytes = (uint32_t)(16 * rz * 16);  // 16 chunks x rz rows x 16 B
    unsigned char *sB = smem;                              // NB x B_BYTES
    unsigned char *sA = smem + NB * B_BYTES;               // NP x plane_bytes
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + NP * plane_bytes);  // load, mma
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int m = tid & (TC_CH - 1);  // this thread's channel in the tile = its TMEM lane
    const int h = tid / TC_CH;        // which half of the k0 outputs it stores
    const int64_t ch0 = (int64_t)blockIdx.x * TC_CH;
    const int qa = blockIdx.y * p.chunk;
    if (qa >= p.rows_out) return;  // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);

    if (warp == 0) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
    }
    // B = realified F0 (K-major): rows n (Re k0 | Im k0), columns k (Re j0 | Im j0)
    for (int e = tid; e < N * K; e += TCC_THREADS) {
        const int n = e / K, k = e - (e / K) * K;
        const int k0 = n & (n0 - 1), j0 = k & (n0 - 1);
        const float2 w = p.om64[((j0 * k0) & (n0 - 1)) << (6 - M0)];  // (C, -S)
        const bool out_im = n >= n0, in_im = k >= n0;
        const float v = (out_im == in_im) ? w.x : (in_im ? -w.y : w.y);
        const uint16_t hi = to_bits<F16>(v);
        const uint32_t off = kmajor_off(n, k, K);
        *reinterpret_cast<uint16_t *>(sB + off) = hi;
        if (NB == 2) *reinterpret_cast<uint16_t *>(sB + B_BYTES + off) = to_bits<F16>(v - from_bits<F16>(hi));
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    if (tid == 0) {
        mbar_expect_tx(&bars[0], NP * plane_bytes);
        for (int pl = 0; pl < NP; ++pl)
            for (int c = 0; c < 16; ++c)
                tma_load_2d(sA + pl * plane_bytes + c * rz * 16, &p.planes[pl], &bars[0], (int)(ch0 + 8 * c), qa);
    }
    ok = __syncthreads_and(mbar_wait(&bars[0], 0, TC_MAX_POLLS));  // block-uniform

    const int n1 = 1 << p.m1;
    constexpr int HK = n0 / 2;  // k0 values per thread: [h HK, (h + 1) HK)
    const int64_t ch = ch0 + m;
    const bool active = ch < p.nch;
    const int64_t q1 = ch >> p.m1, k1 = ch & (n1 - 1);
    float2 *dst = p.out + (int64_t)qa * p.orow + q1 * ((int64_t)n0 * n1) + (int64_t)(h * HK) * n1 + k1;
    const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
    static_assert(n0 >= 16, "each 16-row k-step must lie in one plane");
    const uint32_t a_lbo = 128u;  // K-group stride of A: consecutive 16-byte rows
    const uint32_t a_sbo = (uint32_t)rz * 16u;
    const uint32_t b_lbo = 128u, b_sbo = (uint32_t)(K / 8) * 128u;
    const float out_scale = p.scale / fp16_prescale(p.amax, p.amax_mult);

    // issue all UMMAs of window row i into TMEM buffer i & 1, then commit
    auto issue = [&](int i) {
        const uint32_t d_tmem = tmem + (uint32_t)((i & 1) * N);
        tc_fence_after();
#pragma unroll
        for (int t = 0; t < TERMS; ++t) {
            const int a_set = (t == 2) ? 1 : 0;  // A lo only in the third term
            const int b_set = (t == 1) ? 1 : 0;  // B lo only in the second term
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const int kk = ks * 16;
                const int part = kk / n0;  // 0: Re rows, 1: Im rows
                const int row = i + kk % n0;
                const uint32_t a_addr = sA0 + (uint32_t)((2 * a_set + part) * plane_bytes + row * 16);
                const uint32_t b_addr = sB0 + (uint32_t)(b_set * B_BYTES + ks * 2 * 128);
                umma_f16(d_tmem, smem_desc(a_addr, a_lbo, a_sbo), smem_desc(b_addr, b_lbo, b_sbo), IDESC,
                         (t | ks) != 0);
            }
        }
        umma_commit(&bars[1]);
    };

    // Pipeline: the products of row i+1 run in the other TMEM buffer while row i's epilogue
    // drains.  Row i+1 is issued only after every thread has seen row i's phase complete (the
    // barrier below), so no waiter ever falls two phases behind the parity it waits for; its
    // buffer (i+1)&1 was last read in iteration i-1, before that same barrier.
    const int L = qb - qa;
    if (tid == 0 && ok) issue(0);
    for (int i = 0; i < L && ok; ++i) {
        const bool done = mbar_wait(&bars[1], (uint32_t)(i & 1), TC_MAX_POLLS);
        tc_fence_before();              // orders the previous iteration's TMEM loads
        ok = __syncthreads_and(done);   // block-uniform
        if (!ok) break;
        tc_fence_after();
        if (tid == 0 && i + 1 < L) issue(i + 1);
        // epilogue: this thread's TMEM lane = its channel (warp w reads lanes 32 (w mod 4));
        // columns k0 (Re) and n0 + k0 (Im) for its half of the k0
        const uint32_t lane_addr = tmem + (uint32_t)((i & 1) * N) + ((uint32_t)((warp & 3) * 32) << 16);
        float re[HK], im[HK];
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            float *acc = part ? im : re;
            const uint32_t col = lane_addr + (uint32_t)(part * n0 + h * HK);
            if constexpr (HK >= 16) {
#pragma unroll
                for (int c = 0; c < HK; c += 16) {
                    float v[16];
                    tmem_ld_16(col + c, v);
                    tmem_ld_wait();  // the loaded registers are valid only after the wait
#pragma unroll
                    for (int u = 0; u < 16; ++u) acc[c + u] = v[u];
                }
            } else {
                float v[8];
                tmem_ld_8(col, v);
                tmem_ld_wait();
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = v[u];
            }
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < HK; ++k)
                __stcs(dst + (int64_t)k * n1, make_float2(out_scale * re[k], out_scale * im[k]));
        }
        dst += p.orow;
    }
    if (!ok) {
        // a wait timed out: record it, give in-flight copies and products a last bounded
        // chance to land, then release TMEM
        if (tid == 0) atomicExch(&g_tc_status, 1);
        mbar_wait(&bars[0], 0, 64);
        mbar_wait(&bars[1], 0, 64);
        mbar_wait(&bars[1], 1, 64);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}


// ------------------------------------------------------------------ row DFT on tcgen05
//
// z[r][q1][k1] = sum_j1 x[r][q1 + j1] F1[j1][k1], one product per input row and 128 window
// positions: D (128 x 2n1) = A (128 x K) * B (K x 2n1), A[m][k] = x[r][q1_0 + m + k] (Re x,
// then Im x for complex input; K padded to a multiple of 16 with rows of B that are zero),
// B = realified F1.  A is a Hankel matrix: consecutive positions shift by one element.  As an
// MN-major operand (a core matrix = 8 consecutive positions x 8 consecutive k, one 16-byte
// row per k) its core matrix (m / 8, k / 8) holds x[8 (m/8 + k/8) + (k mod 8) + 0..7] in row
// k mod 8: so the staged row is written eight times, shifted by s = 0..7 elements, unit u
// (16 bytes: x[8u + s .. 8u + s + 7]) of copy s at byte (8u + s) 16, and every core matrix
// is one 128-byte unit row further along M and along K (both descriptor strides 128 B).
// Complex input interleaves the Re and Im unit rows (unit row 2u + part).  The epilogue writes
// z directly as the column pass's operand planes.

constexpr int TCR_ROWS = 8;  // input rows per CTA
constexpr int TCR_TQ = 2;    // threads per position (TMEM lane): A chunks and epilogue slices
constexpr int TCR_ISSUER = TCR_TQ * TC_CH;  // one more warp whose lane 0 issues the UMMAs
constexpr int TCR_THREADS = TCR_ISSUER + 32;

struct TcRowParams {
    const void *x;       // first input row of the band
    int64_t ld;          // input row stride, elements
    int N1, P1, zrows;
    uint16_t *planes;    // [plane][zrows][P1 * n1]
    int64_t plane_elems; // zrows * P1 * n1
    const float *amax;   // per-image fp16 scaling (max |x|; |z| <= n1 * max |x|), or null
    float2 om64[kMaxN];
};

__host__ __device__ constexpr int tcr_K(int M1, bool cplx) {
    return ((cplx ? 2 : 1) << M1) < 16 ? 16 : ((cplx ? 2 : 1) << M1);
}

// A's shifted copies: unit rows per part (positions 0..127 plus K per part, in 8-element units)
// and bytes per operand set
__host__ __device__ constexpr int tcr_units(int M1, bool cplx) {
    return TC_CH / 8 + ((cplx ? (1 << M1) : tcr_K(M1, false)) + 7) / 8;
}
__host__ __device__ constexpr int tcr_copy_bytes(int M1, bool cplx) { return (cplx ? 2 : 1) * tcr_units(M1, cplx) * 128; }

size_t tc_row_smem_bytes(int m1, bool cplx, int terms) {
    const int n1 = 1 << m1, K = tcr_K(m1, cplx), N = 2 * n1, nb = terms == 3 ? 2 : 1;
    const int W = TC_CH + n1;  // staged columns per row (n1 - 1 look-ahead, rounded)
    // staged rows, B (nb sets), A's copies (two buffers of nb sets), barriers and TMEM slot,
    // alignment
    return (size_t)TCR_ROWS * W * (cplx ? 2 : 1) * 4 + (size_t)nb * N * K * 2 +
           (size_t)2 * nb * tcr_copy_bytes(m1, cplx) + 64 + 1024 + 8192;
}

// Pipelined over the CTA's rows: while the tensor core multiplies row r (A buffer and TMEM
// accumulator r mod 2), the threads write row r-1's epilogue and build row r+1's A.  Thread
// (m, h), h < TCR_TQ: position m = TMEM lane; it builds A chunks g = h mod TCR_TQ and stores
// slice h of D's 2 n1 columns (slices of max(16, 2 n1 / TCR_TQ) columns: Re k1 then Im k1).
// A last warp issues the UMMAs, so that issuing them is off the other threads' path.
template <int M1, bool CPLX, int TERMS, bool F16>
__global__ void __launch_bounds__(TCR_THREADS) tc_row_kernel(const __grid_constant__ TcRowParams p) {
    constexpr int n1 = 1 << M1;
    constexpr int K = tcr_K(M1, CPLX);
    constexpr int N = 2 * n1;
    constexpr int KS = K / 16;
    constexpr int NB = TERMS == 3 ? 2 : 1;
    constexpr int W = TC_CH + n1;
    constexpr uint32_t TMEM_COLS = 2 * N < 32 ? 32 : 2 * N;  // two accumulators
    constexpr uint32_t B_BYTES = N * K * 2;
    constexpr int U = tcr_units(M1, CPLX);                    // unit rows per part
    constexpr uint32_t A_BYTES = tcr_copy_bytes(M1, CPLX);    // one set of A's copies
    constexpr uint32_t IDESC = umma_idesc_f16(TC_CH, N, !F16, /*a_mn=*/true, /*b_mn=*/false);
    // A's descriptor strides: along K and along M one unit row (real), two (complex: Re and Im
    // interleaved), except a complex n1 = 8, whose one 16-wide k-step covers Re (k < 8) then
    // Im (k >= 8): its K step goes from the Re unit row to the Im one
    constexpr uint32_t A_SBO = CPLX ? 256u : 128u;
    constexpr uint32_t A_LBO = (CPLX && n1 == 8) ? 128u : A_SBO;
    constexpr int SW = N / TCR_TQ < 16 ? 16 : N / TCR_TQ;  // D columns per epilogue slice
    constexpr int NSL = N / SW;                             // slices: 1 (n1 = 8) or TCR_TQ

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sB = smem;                                   // NB x B_BYTES
    unsigned char *sA = sB + NB * B_BYTES;                      // 2 buffers x NB x A_BYTES (copies)
    float *sx = reinterpret_cast<float *>(sA + 2 * NB * A_BYTES);  // TCR_ROWS x W (x2 complex)
    uint64_t *bar = reinterpret_cast<uint64_t *>(sx + TCR_ROWS * W * (CPLX ? 2 : 1));  // 2 barriers
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = tid & (TC_CH - 1);  // this thread's position in the tile = its TMEM lane
    const int h = tid >> 7;           // 0 .. TCR_TQ - 1; TCR_TQ for the issuing warp
    const bool worker = h < TCR_TQ;
    const int q1_0 = blockIdx.x * TC_CH;
    const int r0 = blockIdx.y * TCR_ROWS;
    if (r0 >= p.zrows) return;  // uniform per block
    const int nrows = min(TCR_ROWS, p.zrows - r0);
    const float pre = F16 ? fp16_prescale(p.amax, (float)n1) : 1.f;

    if (warp == 0) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    // the twiddle table in shared memory: the B build below indexes it per lane
    __shared__ float2 s_om[kMaxN];
    if (tid < kMaxN) s_om[tid] = p.om64[tid];
    __syncthreads();
    // B = realified F1 (K-major): rows n (Re k1 | Im k1), columns k (Re j1 | Im j1 | zero pad)
    for (int e = tid; e < N * K; e += TCR_THREADS) {
        const int n = e / K, k = e - (e / K) * K;
        const int k1 = n & (n1 - 1);
        const bool in_im = CPLX && k >= n1 && k < 2 * n1;
        const bool pad = CPLX ? (k >= 2 * n1) : (k >= n1);
        const int j1 = k & (n1 - 1);
        const float2 w = s_om[((j1 * k1) & (n1 - 1)) << (6 - M1)];  // (C, -S)
        const bool out_im = n >= n1;
        const float v = pad ? 0.f : ((out_im == in_im) ? w.x : (in_im ? -w.y : w.y));
        const uint16_t hi = to_bits<F16>(v);
        const uint32_t off = kmajor_off(n, k, K);
        *reinterpret_cast<uint16_t *>(sB + off) = hi;
        if (NB == 2) *reinterpret_cast<uint16_t *>(sB + B_BYTES + off) = to_bits<F16>(v - from_bits<F16>(hi));
    }
    // stage the CTA's input rows (columns q1_0 .. q1_0 + W - 1; zero beyond the array)
    for (int e = tid; e < nrows * W; e += TCR_THREADS) {
        const int rr = e / W, c = e - (e / W) * W;
        const int col = q1_0 + c;
        if (CPLX) {
            float2 v = make_float2(0.f, 0.f);
            if (col < p.N1) v = reinterpret_cast<const float2 *>(p.x)[(int64_t)(r0 + rr) * p.ld + col];
            sx[(rr * W + c) * 2] = v.x * pre;
            sx[(rr * W + c) * 2 + 1] = v.y * pre;
        } else {
            float v = 0.f;
            if (col < p.N1) v = reinterpret_cast<const float *>(p.x)[(int64_t)(r0 + rr) * p.ld + col];
            sx[rr * W + c] = v * pre;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
    const uint32_t lbo = 128u, sbo = (uint32_t)(K / 8) * 128u;  // B: K-major
    const uint64_t a_desc0 = smem_desc(sA0, A_LBO, A_SBO), b_desc0 = smem_desc(sB0, lbo, sbo);

    const int pos = q1_0 + m;
    const int64_t nch = (int64_t)p.P1 * n1;
    bool ok = true, done = true;
    int issued = 0;  // rows whose UMMAs were committed
    for (int rr = 0; rr <= nrows; ++rr) {
        if (rr < nrows && worker) {
            // A of buffer rr & 1: the shifted copies of input row rr (Re, then Im), unit (u, s)
            // per thread, consecutive threads on consecutive 16-byte slots.  Staged columns
            // past the row (only ever multiplied by B's zero rows, or feeding positions past
            // P1 that are not stored) read as zero.  The buffer's last reader, row rr - 2's
            // UMMAs, completed: every thread waited for them in row rr - 2's epilogue.
            unsigned char *a_buf = sA + (rr & 1) * NB * A_BYTES;
            for (int e = tid; e < (CPLX ? 2 : 1) * U * 8; e += TCR_TQ * TC_CH) {
                const int part = CPLX ? e / (U * 8) : 0;
                const int us = e - part * (U * 8);
                const int u = us >> 3, sh = us & 7;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = 8 * u + sh + j;
                    v[j] = 0.f;
                    if (c < W) v[j] = CPLX ? sx[(rr * W + c) * 2 + part] : sx[rr * W + c];
                }
                const uint32_t off = (uint32_t)((CPLX ? 2 * u + part : u) * 128 + sh * 16);
                uint4 h4, l4;
                split_pair<F16>(v[0], v[1], h4.x, l4.x);
                split_pair<F16>(v[2], v[3], h4.y, l4.y);
                split_pair<F16>(v[4], v[5], h4.z, l4.z);
                split_pair<F16>(v[6], v[7], h4.w, l4.w);
                *reinterpret_cast<uint4 *>(a_buf + off) = h4;
                if (NB == 2) *reinterpret_cast<uint4 *>(a_buf + A_BYTES + off) = l4;
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        // A of row rr is complete; row rr - 2's TMEM reads are done; every wait so far succeeded
        ok = __syncthreads_and(done);
        if (!ok) break;  // block-uniform
        if (rr < nrows) {
            if (tid == TCR_ISSUER) {
                tc_fence_after();
                // descriptors of the other operand tiles: the base descriptors plus the byte
                // offset / 16 (every shared address here is below 2^18, so the 14-bit start
                // field never carries)
                const uint64_t a_base = a_desc0 + (uint64_t)(((rr & 1) * NB * A_BYTES) >> 4);
                const uint32_t d_tmem = tmem + (uint32_t)((rr & 1) * N);
#pragma unroll
                for (int t = 0; t < TERMS; ++t) {
                    const int a_set = (t == 2) ? 1 : 0, b_set = (t == 1) ? 1 : 0;
#pragma unroll
                    for (int ks = 0; ks < KS; ++ks) {
                        // k-step ks = k in [16 ks, 16 ks + 16): its first core matrix's unit row
                        const int k0 = 16 * ks;
                        const int a_row = CPLX ? (n1 == 8 ? 0 : 2 * ((k0 % n1) / 8) + k0 / n1) : k0 / 8;
                        umma_f16(d_tmem, a_base + (uint64_t)((a_set * A_BYTES + a_row * 128) >> 4),
                                 b_desc0 + (uint64_t)((b_set * B_BYTES + ks * 256) >> 4), IDESC, (t | ks) != 0);
                    }
                }
                umma_commit(&bar[rr & 1]);
            }
            issued = rr + 1;
        }
        if (rr >= 1 && worker) {
            // epilogue of row e = rr - 1: its D is accumulator e mod 2, barrier e mod 2 in its
            // (e / 2)-th phase
            const int er = rr - 1;
            // warp-uniform, so that the warp's tcgen05.ld below is never divergent
            done = __all_sync(0xffffffffu, mbar_wait(&bar[er & 1], (uint32_t)((er >> 1) & 1), TC_MAX_POLLS));
            tc_fence_after();
            if (done && h < NSL) {
                const int c0 = h * SW;  // first D column of this slice
                float acc[SW];
#pragma unroll
                for (int c = 0; c < SW; c += 16) {
                    float v[16];
                    tmem_ld_16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((er & 1) * N + c0 + c), v);
                    tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) acc[c + u] = v[u];
                }
                if (pos < p.P1) {
                    // z for this position: each group of 8 D columns is 8 consecutive k1 of one
                    // part (column c: part c / n1, 0 = Re and 1 = Im; k1 = c mod n1) -> planes
                    const int64_t base = (int64_t)(r0 + er) * nch + (int64_t)pos * n1;
#pragma unroll
                    for (int g = 0; g < SW / 8; ++g) {
                        const int cc = c0 + 8 * g;
                        const int part = cc / n1;
                        const int64_t off = base + (cc - part * n1);
                        const float *v = acc + 8 * g;
                        uint4 h4, l4;
                        split_pair<F16>(v[0], v[1], h4.x, l4.x);
                        split_pair<F16>(v[2], v[3], h4.y, l4.y);
                        split_pair<F16>(v[4], v[5], h4.z, l4.z);
                        split_pair<F16>(v[6], v[7], h4.w, l4.w);
                        *reinterpret_cast<uint4 *>(p.planes + part * p.plane_elems + off) = h4;
                        if (TERMS == 3) *reinterpret_cast<uint4 *>(p.planes + (2 + part) * p.plane_elems + off) = l4;
                    }
                }
            }
        }
    }
    if (ok) ok = __syncthreads_and(done);  // the last row's wait (block-uniform: no break)
    if (!ok) {
        // a wait gave up: flag it, give the UMMAs in flight a last bounded wait, then release
        if (tid == 0) atomicExch(&g_tc_status, 1);
        if (issued >= 1) mbar_wait(&bar[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1), 64);
        if (issued >= 2) mbar_wait(&bar[(issued - 2) & 1], (uint32_t)(((issued - 2) >> 1) & 1), 64);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

size_t tc_col_smem_bytes(int m0, int terms, int chunk) {
    const int n0 = 1 << m0;
    const int rz = ((chunk + n0 - 1) + 7) / 8 * 8;
    const int nb = terms == 3 ? 2 : 1, np = terms == 3 ? 4 : 2;
    // + barriers, + 1 KB alignment slack, + 8 KB guard band after the staged tiles
    return (size_t)nb * (2 * n0) * (2 * n0) * 2 + (size_t)np * 16 * rz * 16 + 64 + 1024 + 8192;
}

int tc_col_max_chunk(int m0) { return 256 - (1 << m0) + 1 - 7; }

template <int M0, int TERMS, bool F16>
static cudaError_t launch_tc_col_t(const TcColParams &p, dim3 grid, size_t smem, cudaStream_t s) {
    auto k = tc_col_kernel<M0, TERMS, F16>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, TCC_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tc_col(const TcColArgs &a, cudaStream_t s) {
    if (a.rows_out <= 0) return cudaSuccess;
    if (a.m0 < 4 || a.m0 > kMaxLog2 || a.m1 < 3 || a.m1 > kMaxLog2) return cudaErrorInvalidValue;
    if (a.terms != 1 && a.terms != 3) return cudaErrorInvalidValue;
    const int n0 = 1 << a.m0;
    const int64_t nch = a.P1 << a.m1;
    const int64_t zrows = a.rows_out + n0 - 1;
    const int chunk = (int)std::min<int64_t>(std::min<int64_t>(a.chunk > 0 ? a.chunk : 64, a.rows_out),
                                             tc_col_max_chunk(a.m0));
    const int rz = ((chunk + n0 - 1) + 7) / 8 * 8;
    if (nch % 8 != 0 || zrows > INT32_MAX || (uintptr_t)a.planes % 16 != 0) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    TcColParams p;
    std::memset(&p, 0, sizeof(p));
    const int np = a.terms == 3 ? 4 : 2;
    for (int pl = 0; pl < np; ++pl) {
        cuuint64_t dims[2] = {(cuuint64_t)nch, (cuuint64_t)zrows};
        cuuint64_t strides[1] = {(cuuint64_t)nch * 2};
        cuuint32_t box[2] = {8, (cuuint32_t)rz};
        cuuint32_t estr[2] = {1, 1};
        void *base = static_cast<char *>(a.planes) + (size_t)pl * nch * zrows * 2;
        CUresult r = enc(&p.planes[pl], a.f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    p.out = a.out;
    p.nch = nch;
    p.orow = nch << a.m0;
    p.rows_out = (int)a.rows_out;
    p.chunk = chunk;
    p.rz = rz;
    p.m1 = a.m1;
    p.scale = a.scale;
    p.amax = a.amax;
    p.amax_mult = a.amax_mult;
    for (int j = 0; j < kMaxN; ++j) p.om64[j] = a.om64[j];
    const size_t smem = tc_col_smem_bytes(a.m0, a.terms, chunk);
    dim3 grid((unsigned)((nch + TC_CH - 1) / TC_CH), (unsigned)((a.rows_out + chunk - 1) / chunk));
    if (grid.y > 65535) return cudaErrorInvalidValue;
#define TC_CASE(M_)                                                                                 \
    case M_:                                                                                        \
        if (a.f16) return launch_tc_col_t<M_, 1, true>(p, grid, smem, s);                           \
        return a.terms == 3 ? launch_tc_col_t<M_, 3, false>(p, grid, smem, s)                       \
                            : launch_tc_col_t<M_, 1, false>(p, grid, smem, s);
    switch (a.m0) {
        TC_CASE(4)
        TC_CASE(5)
        TC_CASE(6)
        default:
            return cudaErrorInvalidValue;
    }
#undef TC_CASE
}


template <int M1, bool CPLX, int TERMS, bool F16>
static cudaError_t launch_tc_row_t(const TcRowParams &p, dim3 grid, size_t smem, cudaStream_t s) {
    auto k = tc_row_kernel<M1, CPLX, TERMS, F16>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, TCR_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

template <int M1>
static cudaError_t launch_tc_row_m(const TcRowParams &p, bool cplx, int terms, bool f16, dim3 grid, size_t smem,
                                   cudaStream_t s) {
    if (f16) return cplx ? launch_tc_row_t<M1, true, 1, true>(p, grid, smem, s)
                         : launch_tc_row_t<M1, false, 1, true>(p, grid, smem, s);
    if (terms == 3) return cplx ? launch_tc_row_t<M1, true, 3, false>(p, grid, smem, s)
                                : launch_tc_row_t<M1, false, 3, false>(p, grid, smem, s);
    return cplx ? launch_tc_row_t<M1, true, 1, false>(p, grid, smem, s)
                : launch_tc_row_t<M1, false, 1, false>(p, grid, smem, s);
}

cudaError_t launch_tc_row(const TcRowArgs &a, cudaStream_t s) {
    if (a.zrows <= 0 || a.P1 <= 0) return cudaSuccess;
    if (a.m1 < 3 || a.m1 > kMaxLog2 || (a.terms != 1 && a.terms != 3)) return cudaErrorInvalidValue;
    if (a.zrows > INT32_MAX || a.N1 > INT32_MAX || (uintptr_t)a.planes % 16 != 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if (a.amax) {
        if ((e = cudaMemsetAsync(a.amax, 0, sizeof(float), s)) != cudaSuccess) return e;
        const int64_t n = a.zrows * a.N1;
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
        amax_x_kernel<<<(unsigned)blocks, 256, 0, s>>>(a.x, a.ld, a.zrows, a.N1, a.cplx, a.amax);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    TcRowParams p;
    std::memset(&p, 0, sizeof(p));
    p.x = a.x;
    p.ld = a.ld;
    p.N1 = (int)a.N1;
    p.P1 = (int)a.P1;
    p.zrows = (int)a.zrows;
    p.planes = static_cast<uint16_t *>(a.planes);
    p.plane_elems = a.zrows * (a.P1 << a.m1);
    p.amax = a.amax;
    for (int j = 0; j < kMaxN; ++j) p.om64[j] = a.om64[j];
    const size_t smem = tc_row_smem_bytes(a.m1, a.cplx != 0, a.terms);
    dim3 grid((unsigned)((a.P1 + TC_CH - 1) / TC_CH), (unsigned)((a.zrows + TCR_ROWS - 1) / TCR_ROWS));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    const bool cplx = a.cplx != 0;
    switch (a.m1) {
        case 3: return launch_tc_row_m<3>(p, cplx, a.terms, a.f16, grid, smem, s);
        case 4: return launch_tc_row_m<4>(p, cplx, a.terms, a.f16, grid, smem, s);
        case 5: return launch_tc_row_m<5>(p, cplx, a.terms, a.f16, grid, smem, s);
        case 6: return launch_tc_row_m<6>(p, cplx, a.terms, a.f16, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t tc_status(int *status, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(status, g_tc_status, sizeof(int));
    if (e == cudaSuccess && reset) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int));
    }
    return e;
}

}  // namespace swdft
