// FP32 tree kernels for the 2D sliding window DFT (arXiv 1707.08213, Section 4.2).
//
// Two passes over the two level groups of the tree:
//   row_tree : levels 1..m1 (Eq. rowfswft2d), along dimension 1 of every input row; its
//              level m1 is z[r][q1][k1] = the n1-point DFT of x[r][q1 .. q1+n1-1].
//   col_tree : levels m1+1..m1+m0 (Eq. colfswft2d), along dimension 0 of every channel
//              (q1, k1) of z; its level m0+m1 is the window's 2D DFT, scaled and stored.
// Both walk window positions with SlidingTree (tree_core.cuh), registers only.
//
// z layout: kZPad(n0) = n0/2 padding rows, then rows x P1 x n1 complex64.  The padding lets
// the column pass read its level-0 look-back z[r - n0/2] without a bounds clamp (values
// read there only feed incomplete border trees, which are never stored; only TMA-staged
// walks of n0 <= 8 rows, which start a whole step group early, read it).
//
// Each column-pass warp covers 32 consecutive channels (q1, k1): its z loads and its
// output stores move 256 contiguous bytes per k0 (full 32-byte sectors).  Outputs go out
// with streaming stores so they do not evict z from L2.
#pragma once

#include <cstdint>

#include <cuda.h>

#include "sm100_ptx.cuh"
#include "swdft_internal.h"
#include "tree_core.cuh"

namespace swdft {

// w_64^{-j}, j < 64: the twiddles of every power-of-two length (kernel parameter).
struct Omega64 {
    float2 w[kMaxN];
};

struct RowParams {
    RowGeom g;
    Omega64 om;
};

struct ColParams {
    ColGeom g;
    Omega64 om;
};

template <bool CPLX>
__device__ __forceinline__ float2 load_x(const void *row, int64_t i) {
    if constexpr (CPLX) {
        return __ldg(reinterpret_cast<const float2 *>(row) + i);
    } else {
        return make_float2(__ldg(reinterpret_cast<const float *>(row) + i), 0.f);
    }
}

// Row pass, one block tile.  Thread = (row, residue c, chunk of window columns).  Lanes hold
// the residue in the low B bits, then the row, so the 2^B threads of one row store adjacent
// k1 together.  Tile (row_block, chunk_idx) covers rows row_block * (threads >> B) ... of the
// pass and window columns [chunk_idx * chunk, ...).
template <int M, int B, bool CPLX>
__device__ __forceinline__ void row_tile(const RowGeom &p, int row_block, int chunk_idx,
                                         const float2 *om64) {
    using Tree = SlidingTree<M, B>;
    constexpr int n = 1 << M;
    const int c = threadIdx.x & ((1 << B) - 1);
    const int row = row_block * (blockDim.x >> B) + (threadIdx.x >> B);
    if (row >= p.rows) return;
    const int qa = chunk_idx * p.chunk;
    if (qa >= p.P1) return;
    const int qb = min(qa + p.chunk, p.P1);
    const int steps = (qb - qa) + (n - 1);

    const char *xrow = reinterpret_cast<const char *>(p.x) +
                       (p.r_base + row) * p.ld * (int64_t)(CPLX ? sizeof(float2) : sizeof(float));
    float2 *dst = p.z + (int64_t)row * p.zrow + (int64_t)qa * n + c;

    Tree tree;
    tree.init(c, om64);
    // The walk starts n/2 steps before the chunk's first complete window: level 1 reads level 0
    // n/2 positions back from memory, and the FIFOs of levels 1 .. M-1 hold n/2 - 1 steps, so
    // the first stored output (step n - 1) needs level 1 from step n/2 on; the zeroed FIFOs only
    // feed steps before it.  n/2 is a multiple of the unroll period (FIFO slots keep their
    // step residues).
    static_assert(Tree::kHalf % Tree::kPeriod == 0, "the walk starts on a whole period");
    for (int jb = Tree::kHalf; jb < steps; jb += Tree::kPeriod) {
        static_for<0, Tree::kPeriod>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int p1 = qa + j;  // window end column
                const float2 xp = load_x<CPLX>(xrow, p1);
                const float2 xs = (M >= 1) ? load_x<CPLX>(xrow, max(p1 - Tree::kHalf, 0))
                                           : make_float2(0.f, 0.f);
                float2 o[Tree::kOut];
                tree.template step<J>(xp, xs, o);
                if (j >= n - 1) {
#pragma unroll
                    for (int t = 0; t < Tree::kOut; ++t) dst[t << B] = o[t];
                    dst += n;
                }
            }
        });
    }
}

template <int M, int B, bool CPLX>
__global__ void __launch_bounds__(128) row_tree_kernel(const __grid_constant__ RowParams p) {
    row_tile<M, B, CPLX>(p.g, blockIdx.x, blockIdx.y, p.om.w);
}

// Rows of z a column-pass block stages per step group: the tree's unroll period
// (2^(M-2) steps) or 8, whichever is larger.  Short trees (n0 <= 16) would otherwise reach a
// block barrier every one to four rows with as little fetched ahead; a group of several
// periods keeps each FIFO slot a compile-time register, since every FIFO depth divides it.
__host__ __device__ constexpr int col_group(int M) { return tg_period(M) > 8 ? tg_period(M) : 8; }

// Rows of z staged in shared memory per column-pass block: a ring that holds the level-0
// look-back (n/2 rows) plus the group being computed and the `ahead` groups being fetched,
// rounded up to a power of two.
__host__ __device__ constexpr int col_ring_rows(int M, int ahead = 1) {
    const int look = M >= 1 ? (1 << (M - 1)) : 0;
    // TMA (ahead 2) loads whole groups: its look-back is rounded up to a group
    const int need = (ahead >= 2 ? (look + col_group(M) - 1) / col_group(M) * col_group(M) : look) +
                     (1 + ahead) * col_group(M);
    int r = 1;
    while (r < need) r <<= 1;
    return r;
}

__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// z rows for a column tile come from one of two stages:
//  * ZStageLoad  : cp.async copies of z rows written by the row pass (two-pass form);
//  * ZStageRowDft: the row levels of Eq. rowfswft2d evaluated in the tile itself (fused
//                  form): z never goes to HBM.
// fetch(ring, r_lo, r_hi, CH, ch0, RD) fills ring rows r_lo..r_hi-1; wait() completes it.
struct ZStageLoad {
    static constexpr bool kGroupAligned = false;  // fetches may start on any row
    const float2 *z;
    int64_t nch;
    __device__ __forceinline__ void fetch(float2 *ring, int r_lo, int r_hi, int CH, int64_t ch0, int RD) {
        const int total = (r_hi - r_lo) * CH;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int rr = r_lo + e / CH;
            const int cc = e - (e / CH) * CH;
            const bool ok = ch0 + cc < nch;
            const float2 *src = z + (int64_t)rr * nch + (ok ? ch0 + cc : 0);
            cp_async_8(&ring[(rr & (RD - 1)) * CH + cc], src, ok);
        }
        cp_async_commit();
    }
    __device__ __forceinline__ void wait() { cp_async_wait_all(); }
};

// Row levels of one z row for 32 channels, by one warp.  Channels are (q1, k1) with k1
// fastest, so the warp covers 32 >> M1 window columns q1 (M1 <= 5).  Level t of the tree under
// the window ending at column p needs level t-1 at p and p - s_t (s_t = 2^(M1-t)); for one
// window that is 2^(M1-t) positions x 2^t nodes = n1 values per level, one per lane:
// lane (i, d) holds node i at position p - d.  Each level is two shuffles and one node
// evaluation T = T_{t-1}(p - d - s_t) + W_t^i T_{t-1}(p - d) per lane; level M1 leaves node
// k1 = lane on lane k1, in natural order.
//
// n1 = 64 (M1 = 6): a warp evaluates one whole window column, both 32-channel halves (the
// tile then holds an even number of channel groups).  A level has 64 values, two per lane:
// value e of lane L is flat index l = 2 L + e in the (i, d) layout above.  For levels 1..5, d
// has at least one bit and its lowest bit is e, so both operands of a value sit in the same
// register (e) of the lanes holding l_c = (i mod 2^(t-1)) 2^(7-t) + d and l_c + 2^(6-t): one
// shuffle each.  After level 5 lane L holds node L at p (e = 0) and at p - 1 (e = 1): level
// 6's nodes L and 32 + L need just those two, in the lane's own registers.  Same nodes,
// operands and operation order as the row pass's tree, so z is bit for bit the two-pass
// form's.
template <int M1, bool CPLX>
struct ZStageRowDft {
    static constexpr bool kGroupAligned = false;  // fetches may start on any row
    const void *x;      // first input row of the band
    int64_t ld;
    int zrows;          // z rows that exist (band rows + n0 - 1)
    int P1;
    // this lane's twiddle per level (M1 <= 5); for M1 = 6, per level 1..5 and value, then
    // level 6's W^lane and W^(32 + lane)
    float2 w[M1 == 6 ? 12 : (M1 > 0 ? M1 : 1)];

    __device__ __forceinline__ void init(const float2 *om64) {
        if constexpr (M1 == 6) {
            const int lane = threadIdx.x & 31;
#pragma unroll
            for (int t = 1; t <= 5; ++t)
#pragma unroll
                for (int e = 0; e < 2; ++e) w[2 * (t - 1) + e] = om64[((2 * lane + e) >> (6 - t)) << (6 - t)];
            w[10] = om64[lane];
            w[11] = om64[32 + lane];
        } else {
            const int l = threadIdx.x & ((1 << M1) - 1);
#pragma unroll
            for (int t = 1; t <= M1; ++t) {
                const int i = l >> (M1 - t);
                w[t - 1] = om64[i << (6 - t)];
            }
        }
    }

    __device__ __forceinline__ float2 load(int r, int64_t col) const {
        if constexpr (CPLX)
            return __ldg(reinterpret_cast<const float2 *>(x) + (int64_t)r * ld + col);
        else
            return make_float2(__ldg(reinterpret_cast<const float *>(x) + (int64_t)r * ld + col), 0.f);
    }

    // n1 = 64: window column q1 of z row r; lane L returns nodes L (lo) and 32 + L (hi)
    __device__ __forceinline__ void row_dft64(int r, int64_t q1, float2 &lo, float2 &hi) const {
        const int lane = threadIdx.x & 31;
        {
            float2 v[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (r >= 0 && r < zrows && q1 < P1) {  // level 0 at flat index d = 2 L + e: x at p - d
                const int64_t p = q1 + 63;
                v[0] = load(r, p - 2 * lane);
                v[1] = load(r, p - 2 * lane - 1);
            }
#pragma unroll
            for (int t = 1; t <= 5; ++t) {
                float2 nv[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int l = 2 * lane + e;
                    const int i = l >> (6 - t), d = l & ((1 << (6 - t)) - 1);
                    const int lc = ((i & ((1 << (t - 1)) - 1)) << (7 - t)) | d;  // node i mod 2^(t-1), offset d
                    const float cx = __shfl_sync(0xffffffffu, v[e].x, lc >> 1);
                    const float cy = __shfl_sync(0xffffffffu, v[e].y, lc >> 1);
                    const float sx = __shfl_sync(0xffffffffu, v[e].x, (lc >> 1) + (1 << (5 - t)));  // offset d + s_t
                    const float sy = __shfl_sync(0xffffffffu, v[e].y, (lc >> 1) + (1 << (5 - t)));
                    nv[e] = c_add(make_float2(sx, sy), c_mul(w[2 * (t - 1) + e], make_float2(cx, cy)));
                }
                v[0] = nv[0];
                v[1] = nv[1];
            }
            lo = c_add(v[1], c_mul(w[10], v[0]));
            hi = c_add(v[1], c_mul(w[11], v[0]));
        }
    }

    __device__ __forceinline__ float2 row_dft(int r, int64_t ch0) const {
        const int lane = threadIdx.x & 31;
        {
            const int l = lane & ((1 << M1) - 1);
            const int base = lane - l;
            const int64_t q1 = (ch0 >> M1) + (lane >> M1);
            float2 v = make_float2(0.f, 0.f);
            if (r >= 0 && r < zrows && q1 < P1) v = load(r, q1 + (1 << M1) - 1 - l);  // level 0 on lane d: x at p - d
#pragma unroll
            for (int t = 1; t <= M1; ++t) {
                const int i = l >> (M1 - t), d = l & ((1 << (M1 - t)) - 1);
                const int src = base + ((i & ((1 << (t - 1)) - 1)) << (M1 - t + 1)) + d;  // node i mod 2^(t-1), offset d
                const float cx = __shfl_sync(0xffffffffu, v.x, src);
                const float cy = __shfl_sync(0xffffffffu, v.y, src);
                const float sx = __shfl_sync(0xffffffffu, v.x, src + (1 << (M1 - t)));  // offset d + s_t
                const float sy = __shfl_sync(0xffffffffu, v.y, src + (1 << (M1 - t)));
                v = c_add(make_float2(sx, sy), c_mul(w[t - 1], make_float2(cx, cy)));
            }
            return v;
        }
    }

    __device__ __forceinline__ void fetch(float2 *ring, int r_lo, int r_hi, int CH, int64_t ch0, int RD) {
        const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        const int lane = threadIdx.x & 31;
        if constexpr (M1 == 6) {
            const int cols = CH >> 6;  // whole window columns of the tile (CH a multiple of 64)
            for (int e = warp; e < (r_hi - r_lo) * cols; e += nwarp) {
                const int rr = r_lo + e / cols, wc = e - (e / cols) * cols;
                float2 lo, hi;
                row_dft64(rr, (ch0 >> 6) + wc, lo, hi);
                float2 *dst = ring + (rr & (RD - 1)) * CH + wc * 64 + lane;
                dst[0] = lo;
                dst[32] = hi;
            }
        } else {
            const int groups = CH >> 5;
            for (int e = warp; e < (r_hi - r_lo) * groups; e += nwarp) {
                const int rr = r_lo + e / groups, g = e - (e / groups) * groups;
                ring[(rr & (RD - 1)) * CH + g * 32 + lane] = row_dft(rr, ch0 + g * 32);
            }
        }
    }
    __device__ __forceinline__ void wait() {}
};

// Column pass, one block tile.  Thread = (channel ch = q1*n1 + k1, residue c, chunk of
// window rows).  Warp w of a block takes residue w mod 2^B (uniform per warp) and channel
// group w / 2^B.  The tile's z rows reach a shared-memory ring AHEAD step groups ahead of use
// (copied or computed by the stage; stage.wait() completes the oldest fetch still in flight);
// all residue warps read the same staged rows.  One __syncthreads per step group; the tile
// ends with a barrier, so the ring is free for the next tile.
template <int M, int B, int AHEAD = 1, class Stage>
__device__ __forceinline__ void col_tile_impl(const ColGeom &p, int64_t ch_block, int chunk_idx,
                                              const float2 *om64, float2 *ring, Stage &stage,
                                              int64_t slice = 0) {
    using Tree = SlidingTree<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    constexpr int kP = col_group(M);  // steps per staged group, a multiple of Tree::kPeriod
    constexpr int kH = Tree::kHalf;
    constexpr int RD = col_ring_rows(M, AHEAD);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int c = warp & (R - 1);
    const int CH = 32 * p.groups;                       // channels of this tile
    const int my = (warp >> B) * 32 + lane;             // this thread's channel in the tile
    const int64_t ch0 = ch_block * CH;
    const int64_t ch = ch0 + my;
    const int qa = chunk_idx * p.chunk;
    if (qa >= p.rows_out) return;                       // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const int steps = (qb - qa) + (n - 1);
    const int zr_end = qb + n - 1;                      // one past the last z row used
    const bool active = ch < p.nch;

    const int n1 = 1 << p.m1;
    const int64_t q1 = ch >> p.m1;
    const int64_t k1 = ch & (n1 - 1);
    const int kstride = R * n1;  // elements between outputs t and t+1 (k0 step 2^B)
    // First step of the walk: n/2 (as in row_tile), rounded down to whole step groups for a
    // stage whose every fetch must start on a group (TMA boxes; n/2 for n0 >= 16 anyway).  n/2
    // is a multiple of the unroll period, so FIFO slots keep their step residues.
    constexpr int kJ0 = Stage::kGroupAligned ? (kH / kP) * kP : kH;
    float2 *dst = p.out + slice * p.oslice + (int64_t)qa * p.orow + q1 * ((int64_t)n * n1) +
                  (int64_t)c * n1 + k1;
    const float s = p.scale;

    Tree tree;
    tree.init(c, om64);
    stage.fetch(ring, qa + kJ0 - kH, min(qa + kJ0 + kP, zr_end), CH, ch0, RD);
#pragma unroll
    for (int a = 1; a < AHEAD; ++a)
        if (kJ0 + a * kP < steps)
            stage.fetch(ring, qa + kJ0 + a * kP, min(qa + kJ0 + (a + 1) * kP, zr_end), CH, ch0, RD);
    stage.wait();
    __syncthreads();
    for (int jb = kJ0; jb < steps; jb += kP) {
        if (jb + AHEAD * kP < steps)
            stage.fetch(ring, qa + jb + AHEAD * kP, min(qa + jb + (AHEAD + 1) * kP, zr_end), CH, ch0, RD);
        static_for<0, kP>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if (j < steps) {
                const int zr = qa + j;  // z row = window end row, relative to the band
                const float2 xp = ring[(zr & (RD - 1)) * CH + my];
                const float2 xs = (M >= 1) ? ring[((zr - kH) & (RD - 1)) * CH + my] : make_float2(0.f, 0.f);
                float2 o[Tree::kOut];
                tree.template step<J>(xp, xs, o);
                if (j >= n - 1 && active) {
#pragma unroll
                    for (int t = 0; t < Tree::kOut; ++t) __stcs(dst + t * kstride, c_scale(s, o[t]));
                    dst += p.orow;
                }
            }
        });
        stage.wait();
        __syncthreads();
    }
}

template <int M, int B>
__device__ __forceinline__ void col_tile(const ColGeom &p, int64_t ch_block, int chunk_idx,
                                         const float2 *om64, float2 *ring, int64_t slice = 0) {
    ZStageLoad stage{p.z + slice * p.zslice, p.nch};
    col_tile_impl<M, B>(p, ch_block, chunk_idx, om64, ring, stage, slice);
}

// grid: x = 32-channel groups, y = chunks of window rows, z = slices (kD passes; 1 in 2D).
// Two resident 256-thread blocks per SM cap a thread at 128 registers; the 64-point tree
// (M = 6) needs about 150 and spilled under that cap, so it asks for one block (the pass
// alone measured 5-6% faster on 512x512 and 1024x1024 with 64x16 windows).  The fused
// kernel keeps two blocks: with one, 1024x1024 with 64x16 windows went from 1.37 to 1.56 ms.
template <int M, int B>
__global__ void __launch_bounds__(256, (M >= 6 ? 1 : 2)) col_tree_kernel(const __grid_constant__ ColParams p) {
    extern __shared__ float2 ring[];  // col_ring_rows(M) x (32 * groups)
    col_tile<M, B>(p.g, blockIdx.x, blockIdx.y, p.om.w, ring, blockIdx.z);
}

// z rows by TMA (two-pass form of a single array): z is described, from its first padding
// row, as a 2D tensor [rows][nch] of 8-byte elements, and a step group of kP z rows is one
// tiled load of a box of CH channels x kP rows (channels past nch and rows outside z read as
// zero), issued by thread 0 and completing on the mbarrier of its fetch.  The tile's chunk
// starts on a multiple of kP and its look-back is rounded up to whole groups, so every box
// starts on a multiple of kP and lands in kP consecutive rows of the ring (a multiple of kP
// rows long); rows a box carries beyond those asked for are never read.  The tile runs two
// step groups ahead.  Waits are bounded: a wait that gives up records it in g_col_tma_status and the block
// carries on (its outputs are then wrong; nothing hangs).
constexpr uint32_t kColTmaPolls = 2000;  // ~1 ms per poll at most
static __device__ int g_col_tma_status;  // one word per translation unit (no relocatable device code)

// Fetch f completes on barrier f mod kColTmaBars, phase f / kColTmaBars; with the tile
// kColTmaAhead groups ahead, a barrier is re-armed only after its previous fetch was waited for.
constexpr int kColTmaAhead = 2;
constexpr int kColTmaBars = kColTmaAhead + 1;
template <int kP>
struct ZStageTma {
    static constexpr bool kGroupAligned = true;  // every box starts on a whole step group
    const CUtensorMap *map;
    int pad;            // padding rows in front of z (tensor row of z row r = r + pad)
    uint64_t *bar;      // kColTmaBars mbarriers in shared memory
    int k = 0;          // fetches issued so far
    int w = 0;          // fetches waited for so far
    // rows [r_lo, r_hi) widened to whole groups [floor(r_lo / kP) kP, ceil(r_hi / kP) kP)
    __device__ __forceinline__ void fetch(float2 *ring, int r_lo, int r_hi, int CH, int64_t ch0, int RD) {
        if (threadIdx.x == 0) {
            const int g0 = r_lo >= 0 ? r_lo / kP : -((kP - 1 - r_lo) / kP);
            const int g1 = (r_hi + kP - 1) / kP;
            uint64_t *b = &bar[k % kColTmaBars];
            fence_proxy_async_smem();  // the rows refilled here were last read by generic loads
            mbar_expect_tx(b, (uint32_t)((g1 - g0) * kP * CH * sizeof(float2)));
            for (int g = g0; g < g1; ++g)
                tma_load_2d(ring + ((g * kP) & (RD - 1)) * CH, map, b, (int)ch0, g * kP + pad);
        }
        ++k;
    }
    // completes the oldest fetch still in flight
    __device__ __forceinline__ void wait() {
        if (w >= k) return;
        const int f = w++;
        if (!mbar_wait(&bar[f % kColTmaBars], (uint32_t)(f / kColTmaBars) & 1u, kColTmaPolls))
            atomicExch(&g_col_tma_status, 1);
    }
};

struct ColTmaParams {
    CUtensorMap zmap;   // z from its first padding row: [pad + rows][nch], 8-byte elements
    ColGeom g;          // g.z unused
    int pad;
    Omega64 om;
};

template <int M, int B>
__global__ void __launch_bounds__(256, (M >= 6 ? 1 : 2)) col_tree_tma_kernel(const __grid_constant__ ColTmaParams p) {
    extern __shared__ __align__(128) unsigned char col_smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(col_smem);       // kColTmaBars mbarriers
    float2 *ring = reinterpret_cast<float2 *>(col_smem + 128);    // col_ring_rows(M, 2) x (32 * groups)
    if (threadIdx.x == 0) {
        for (int b = 0; b < kColTmaBars; ++b) mbar_init(&bar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    ZStageTma<col_group(M)> stage{&p.zmap, p.pad, bar};
    col_tile_impl<M, B, kColTmaAhead>(p.g, blockIdx.x, blockIdx.y, p.om.w, ring, stage);
}

// Fused form: both level groups in one kernel, x in, window DFTs out (n1 <= 64).
struct FusedParams {
    ColGeom g;          // g.z unused
    const void *x;      // first input row of the band
    int64_t ld;
    int zrows, P1;
    Omega64 om;
};

template <int M0, int B, int M1, bool CPLX>
__global__ void __launch_bounds__(256, 2) fused_tree_kernel(const __grid_constant__ FusedParams p) {
    extern __shared__ float2 ring[];
    ZStageRowDft<M1, CPLX> stage;
    stage.x = p.x;
    stage.ld = p.ld;
    stage.zrows = p.zrows;
    stage.P1 = p.P1;
    stage.init(p.om.w);
    col_tile_impl<M0, B>(p.g, blockIdx.x, blockIdx.y, p.om.w, ring, stage);
}

template <int M, int B>
void row_launch_mb(const RowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s);
template <int M0, int B>
void fused_launch_mb(const FusedParams &p, int m1, int cplx, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
void col_launch_mb(const ColParams &p, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
void col_tma_launch_mb(const ColTmaParams &p, dim3 g, dim3 b, cudaStream_t s);
template <int M>
cudaError_t col_tma_status_mb(int *status, bool reset);  // the g_col_tma_status of M's unit
template <int M, int B>
int col_blocks_per_sm(int threads, int groups);

#define SWDFT_ROW_INSTANTIATE(M_, B_)                                                        \
    template <>                                                                              \
    void row_launch_mb<M_, B_>(const RowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s) { \
        if (cplx)                                                                            \
            row_tree_kernel<M_, B_, true><<<g, b, 0, s>>>(p);                                \
        else                                                                                 \
            row_tree_kernel<M_, B_, false><<<g, b, 0, s>>>(p);                               \
    }

#define SWDFT_COL_INSTANTIATE(M_, B_)                                                     \
    template <>                                                                           \
    void col_launch_mb<M_, B_>(const ColParams &p, dim3 g, dim3 b, cudaStream_t s) {      \
        const size_t smem = sizeof(float2) * col_ring_rows(M_) * 32 * p.g.groups;          \
        col_tree_kernel<M_, B_><<<g, b, smem, s>>>(p);                                    \
    }                                                                                     \
    template <>                                                                           \
    void col_tma_launch_mb<M_, B_>(const ColTmaParams &p, dim3 g, dim3 b, cudaStream_t s) { \
        const size_t smem = 128 + sizeof(float2) * col_ring_rows(M_, kColTmaAhead) * 32 * p.g.groups; \
        col_tree_tma_kernel<M_, B_><<<g, b, smem, s>>>(p);                                \
    }                                                                                     \
    template <>                                                                           \
    int col_blocks_per_sm<M_, B_>(int threads, int groups) {                              \
        int nb = 0;                                                                       \
        const size_t smem = sizeof(float2) * col_ring_rows(M_) * 32 * groups;             \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, col_tree_kernel<M_, B_>,   \
                                                          threads, smem) != cudaSuccess)  \
            return 0;                                                                     \
        return nb;                                                                        \
    }

#define SWDFT_FUSED_INSTANTIATE(M_, B_)                                                          \
    template <>                                                                                  \
    void fused_launch_mb<M_, B_>(const FusedParams &p, int m1, int cplx, dim3 g, dim3 b,         \
                                 cudaStream_t s) {                                               \
        const size_t smem = sizeof(float2) * col_ring_rows(M_) * 32 * p.g.groups;               \
        switch (m1 * 2 + cplx) {                                                                 \
            case 0: fused_tree_kernel<M_, B_, 0, false><<<g, b, smem, s>>>(p); break;            \
            case 1: fused_tree_kernel<M_, B_, 0, true><<<g, b, smem, s>>>(p); break;             \
            case 2: fused_tree_kernel<M_, B_, 1, false><<<g, b, smem, s>>>(p); break;            \
            case 3: fused_tree_kernel<M_, B_, 1, true><<<g, b, smem, s>>>(p); break;             \
            case 4: fused_tree_kernel<M_, B_, 2, false><<<g, b, smem, s>>>(p); break;            \
            case 5: fused_tree_kernel<M_, B_, 2, true><<<g, b, smem, s>>>(p); break;             \
            case 6: fused_tree_kernel<M_, B_, 3, false><<<g, b, smem, s>>>(p); break;            \
            case 7: fused_tree_kernel<M_, B_, 3, true><<<g, b, smem, s>>>(p); break;             \
            case 8: fused_tree_kernel<M_, B_, 4, false><<<g, b, smem, s>>>(p); break;            \
            case 9: fused_tree_kernel<M_, B_, 4, true><<<g, b, smem, s>>>(p); break;             \
            case 10: fused_tree_kernel<M_, B_, 5, false><<<g, b, smem, s>>>(p); break;           \
            case 11: fused_tree_kernel<M_, B_, 5, true><<<g, b, smem, s>>>(p); break;            \
            case 12:                                                                             \
                if constexpr (M_ <= 5) fused_tree_kernel<M_, B_, 6, false><<<g, b, smem, s>>>(p); \
                break;                                                                           \
            case 13:                                                                             \
                if constexpr (M_ <= 5) fused_tree_kernel<M_, B_, 6, true><<<g, b, smem, s>>>(p); \
                break;                                                                           \
            default: break;                                                                      \
        }                                                                                        \
    }

// This unit's g_col_tma_status (read and reset by swdft2d_check_device).
#define SWDFT_COL_TMA_STATUS(M_)                                                          \
    template <>                                                                           \
    cudaError_t col_tma_status_mb<M_>(int *status, bool reset) {                          \
        cudaError_t e = cudaMemcpyFromSymbol(status, g_col_tma_status, sizeof(int));      \
        if (e == cudaSuccess && reset && *status != 0) {                                  \
            const int zero = 0;                                                           \
            e = cudaMemcpyToSymbol(g_col_tma_status, &zero, sizeof(int));                 \
        }                                                                                 \
        return e;                                                                         \
    }

// (M, B) pairs built: B <= min(M, 3), and B >= 2 for 64-point trees (fewer threads per tree
// would need more registers than there are; launchers raise B to 2 there)
#define SWDFT_MB_CASES(F)                                                              \
    F(0, 0) F(1, 0) F(1, 1) F(2, 0) F(2, 1) F(2, 2) F(3, 0) F(3, 1) F(3, 2) F(3, 3)     \
    F(4, 0) F(4, 1) F(4, 2) F(4, 3) F(5, 0) F(5, 1) F(5, 2) F(5, 3) F(6, 2) F(6, 3)

__host__ __device__ constexpr int clamp_split(int M, int B) {
    return B < 0 ? 0 : (B > M ? M : (B > 3 ? 3 : (M >= 6 && B < 2 ? 2 : B)));
}

}  // namespace swdft
