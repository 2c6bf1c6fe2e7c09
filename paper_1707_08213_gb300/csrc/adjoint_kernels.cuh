// Adjoint (A^H) kernels of the 2D sliding window DFT: the transposed tree of Section 4.2,
// i.e. the overlap-add of every window's inverse DFT of the upstream gradient G.
//
// The forward map is A = C R (row levels R: x -> z, then column levels C: z -> a, each a
// sliding transform along one axis), so A^H = R^H C^H, again two passes:
//   adj_col : per channel (q1, k1), walk z rows downwards with SlidingTreeAdjoint along
//             dimension 0:  gz[r][q1][k1] = c * sum_j0 sum_k0 G[r-j0][q1][k0][k1] w_{n0}^{+j0 k0}
//   adj_row : per z row, walk columns downwards along dimension 1:
//             gx[r][p1] = sum_j1 sum_k1 gz[r][p1-j1][k1] w_{n1}^{+j1 k1}   (real part for real x)
// gz uses the same workspace as the forward pass's z (rows x P1 x n1 complex64).
//
// adj_col splits the work by WINDOW rows: chunk i takes windows q0 in [qa, qb) and reads
// those rows of G exactly once (G is the large operand: n0 times gz).  Its outputs cover z
// rows [qa, qb + n0 - 2]; rows >= qb are shared with chunk i+1, so chunk i writes them to a
// side buffer, side[i][r - qb][ch] (n0-1 rows per chunk boundary), and adj_fold then adds
// them to gz rows [qb, qb + n0 - 2].  No atomics: the result is deterministic.  adj_row
// stages gz rows through shared memory, GS steps at a time.
//
// adj_row holds the residue c in a lane's low B bits (row above), adj_col in the high bits
// (channel below).  Either way the 2^B partials of one output are reduced with shuffles and
// the c = 0 lanes store.  G is read once, coalesced.
#pragma once

#include <algorithm>
#include <cstdint>

#include "swdft_internal.h"
#include "adjoint_core.cuh"
#include "sm100_ptx.cuh"

namespace swdft {

// Per array (grid z) pointers: arrays of one shape share a launch.
struct AdjRowParams {
    const float2 *gz[kAdjZ];    // zrows x P1 x n1
    void *gx[kAdjZ];            // zrows rows of N1 elements (row stride ld_out)
    int64_t ld_out;
    int zrows;
    int N1, P1;
    int chunk;         // output columns per thread (plus n1 - 1 warm-up steps)
    float2 om64[kMaxN];  // w_64^{-j}: every power-of-two length's twiddles
};

struct AdjFoldParams {
    float2 *gz[kAdjZ];
    const float2 *side[kAdjZ];
    int64_t nch;       // P1 * n1
    int64_t per_row;   // (n0 - 1) * nch: side values per chunk boundary
    int64_t total;     // (chunks - 1) * per_row
    int chunk;         // window rows per adj_col chunk
    int pairs;         // add 16-byte pieces (nch even, gz and side 16-byte aligned)
};

template <int R>
__device__ __forceinline__ float2 reduce_residues(float2 v) {
#pragma unroll
    for (int off = 1; off < R; off <<= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    return v;
}

__host__ __device__ constexpr int adj_col_channels(int B) { return 128 >> B; }

// G is read once: its lines are marked evict-first in L2, so that the gz rows this pass
// writes (n0 times smaller) are still in L2 when adj_row reads them.
__device__ __forceinline__ uint64_t adj_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void adj_cp_async_8(void *smem, const void *gmem, bool valid, uint64_t pol) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2, %3;\n" ::"r"(dst), "l"(gmem),
                 "r"(valid ? 8 : 0), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void adj_cp_async_16_hint(void *smem, const void *gmem, uint64_t pol) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(gmem), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void adj_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void adj_cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void adj_cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void adj_cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------------------------
// Staging of G for adj_col (adj_col_ring_kernel below).
//
// Per step (one window row q0), a block's CH = 128 >> B channels need n0 values each: in G's
// layout [q0][q1][k0][k1] those are, when n1 <= CH, one contiguous run (the block's whole
// q1 groups), and when n1 > CH, n0 runs of CH values (one per k0).  They go to a ring of
// kAdjStages stages of kAdjGS(M) steps in shared memory.
//
// Lanes hold the residue in their HIGH bits (lane = c * (32 >> B) + channel), so a half-warp
// (the unit of a 64-bit shared-memory access) reads consecutive channels of one or two
// residues; the host picks the staging layout (AdjColLayout) that keeps those reads free of
// bank conflicts where it can: one contiguous run, q1 groups separated by padding, or one
// padded run per k0.  Thread (c, channel ch) finds its value of k0 = c + 2^B t at
//     slot[(ch >> lw) * gs + (ch & (2^lw - 1)) + k0 * ks].
// ------------------------------------------------------------------------------------
constexpr int kAdjStages = 2;
__host__ __device__ constexpr int kAdjGS(int M) { return M >= 4 ? 2 : 32 >> M; }  // steps per stage

// Staging layout of one step (see above).  mode 0: one run of CHv * n0 values (n1 <= CH);
// mode 1: one run of n0 * n1 values per q1 group, groups gs apart (n1 < CH); mode 2: one run
// of CH values per k0, runs ks apart (n1 >= CH).  slot = values per staged step.
struct AdjColLayout {
    int mode = 0, lw = 0, gs = 0, ks = 0, slot = 0;
};

// Largest number of distinct 8-byte words that one half-warp's read of a step maps to one
// bank pair (1 = conflict-free), for warp 0 (every warp's pattern is a translate of it).
inline int adj_col_conflicts(int M, int B, const AdjColLayout &L) {
    const int R = 1 << B, CPW = 32 >> B, n = 1 << M, W = 1 << L.lw;
    int worst = 1;
    for (int t = 0; t < n / R; ++t)
        for (int h = 0; h < 2; ++h) {
            int addr[16], cnt[16] = {};
            for (int l = 0; l < 16; ++l) {
                const int lane = 16 * h + l, c = lane / CPW, ch = lane % CPW;
                addr[l] = (ch >> L.lw) * L.gs + (ch & (W - 1)) + (c + R * t) * L.ks;
            }
            for (int l = 0; l < 16; ++l) {
                bool dup = false;
                for (int e = 0; e < l; ++e) dup = dup || addr[e] == addr[l];
                if (!dup) worst = std::max(worst, ++cnt[addr[l] & 15]);
            }
        }
    return worst;
}

// The layout for window side 2^M (split B) and n1 = 2^m1: fewest bank conflicts, then fewest
// runs per step, then the smallest slot; padded q1 groups only when one run would read with
// more than 2-way conflicts (their larger ring costs a resident block: measured slower on
// 1024x1024 with 8x8 windows).  Paddings are even (runs stay 16-byte aligned).
inline AdjColLayout adj_col_layout(int M, int B, int m1) {
    const int n = 1 << M, n1 = 1 << m1, CH = 128 >> B;
    AdjColLayout best;
    int best_cf = 1 << 30, best_runs = 1 << 30;
    auto consider = [&](const AdjColLayout &L, int runs) {
        const int cf = adj_col_conflicts(M, B, L);
        if (cf < best_cf || (cf == best_cf && (runs < best_runs || (runs == best_runs && L.slot < best.slot)))) {
            best = L;
            best_cf = cf;
            best_runs = runs;
        }
    };
    if (n1 <= CH) consider(AdjColLayout{0, m1, n * n1, n1, CH * n}, 1);
    if (n1 < CH && best_cf > 2)
        for (int pad = 2; pad <= 30; pad += 2)
            consider(AdjColLayout{1, m1, n * n1 + pad, n1, (CH >> m1) * (n * n1 + pad)}, CH >> m1);
    if (n1 >= CH) {
        int lw = 0;
        while ((1 << lw) < CH) ++lw;
        for (int pad = 0; pad <= 30; pad += 2) consider(AdjColLayout{2, lw, 0, CH + pad, n * (CH + pad)}, n);
    }
    return best;
}

// Shared memory of one block: 128 bytes, then the ring.
__host__ __device__ constexpr size_t adj_col_smem(int M, int slot) {
    return 128 + sizeof(float2) * (size_t)kAdjStages * kAdjGS(M) * (size_t)slot;
}

// ------------------------------------------------------------------------------------
// adj_col_ring_kernel: the column adjoint with the staging above.
//
// All 128 threads fill the ring with cp.async, 16 bytes (two adjacent channels) per copy, or
// 8 bytes when G is not 16-byte aligned or n1 = 1: a thread issues CH * n0 / 256 copies per
// step (n0 / 2^(B+1)), each two adds from its last.  At each stage boundary a thread waits for
// its own copies of the stage (cp.async.wait_group), one block barrier makes every thread's
// copies visible and frees the slot read in the previous stage, and the stage kAdjStages - 1
// ahead is started into that slot.  No spin-waits.  (A form in which one warp issued
// cp.async.bulk copies completing on mbarriers measured slower: its per-stage bookkeeping
// cost more than the per-thread copies.)
// ------------------------------------------------------------------------------------
struct AdjColRingParams {
    const float2 *G[kAdjZ];
    float2 *gz[kAdjZ];
    float2 *side[kAdjZ];
    int64_t nch;
    int rows_out, chunk, m1;
    int q16;           // 16-byte copies (G 16-byte aligned and n1 >= 2), else 8-byte
    float scale;
    AdjColLayout L;
    float2 om64[kMaxN];
};

template <int M, int B>
__global__ void __launch_bounds__(128, (M <= 4 ? 5 : (M == 5 ? 3 : 1))) adj_col_ring_kernel(
    const __grid_constant__ AdjColRingParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    constexpr int R = 1 << B;
    constexpr int n = 1 << M;
    constexpr int CH = adj_col_channels(B);
    constexpr int CPW = 32 >> B;          // channels per warp
    constexpr int GS = kAdjGS(M);
    constexpr int NS = kAdjStages;
    constexpr int UNR = Tree::kPeriod > GS ? Tree::kPeriod : GS;  // both powers of two
    // The last n/2 drain steps read the level-1 FIFO alone (SlidingTreeAdjoint::tail) for
    // n0 = 16 and 64, where that measured faster (512x512 64x16: 0.97 -> 0.50 ms, 16x16 and
    // 16x64 2-3%); n0 = 32 measured 4% slower with it and n0 <= 8 has at most 4 such steps.
    constexpr bool kTail = M == 4 || M == 6;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *ring = reinterpret_cast<float2 *>(smem_raw + 128);  // [NS][GS][slot]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane / CPW;
    const int chl = warp * CPW + (lane & (CPW - 1));  // this thread's channel within the block
    const int64_t ch0 = (int64_t)blockIdx.x * CH;
    const int64_t ch = ch0 + chl;
    const bool active = ch < p.nch;
    const int qa = blockIdx.y * p.chunk;  // windows [qa, qb) of this chunk
    if (qa >= p.rows_out) return;         // uniform per block
    const int qb = min(qa + p.chunk, p.rows_out);
    const bool last = qb == p.rows_out;
    const int p_hi = qb + n - 2;
    const int nwin = qb - qa;
    const int steps = nwin + n - 1;
    const int ngroups = (nwin + GS - 1) / GS;  // stages holding at least one row of G
    const float s = p.scale;
    const int slot = p.L.slot;

    const AdjColLayout L = p.L;
    const int n1 = 1 << p.m1;
    const int chv = (int)(p.nch - ch0 < CH ? p.nch - ch0 : CH);  // channels present: even when n1 >= 2
    const int64_t grow = p.nch * n;
    const int64_t gbase = (ch0 >> p.m1) * n * n1 + (ch0 & (n1 - 1));  // the block's first channel, k0 = 0
    // Copies: thread i owns one channel pair (16-byte pieces; one channel with 8-byte pieces)
    // and the k0 = i / pairs + KS * t of every step, so each of its copies is two adds away
    // from the last: in G a step's (k0, channel) is at gbase + (ch >> m1) n n1 + k0 n1 +
    // (ch & (n1 - 1)), in the staged step at (ch >> lw) gs + (ch & (2^lw - 1)) + k0 ks.
    const bool q16 = p.q16;
    const int cl = q16 ? 2 * (threadIdx.x % (CH / 2)) : threadIdx.x % CH;  // first channel copied
    const int k0f = q16 ? threadIdx.x / (CH / 2) : threadIdx.x / CH;        // first k0 copied
    const bool okf = cl < chv && k0f < n;
    const float2 *gsrc = p.G[blockIdx.z] + gbase + (cl >> p.m1) * n * n1 + (cl & (n1 - 1)) + (int64_t)k0f * n1;
    const int sdst = (cl >> L.lw) * L.gs + (cl & ((1 << L.lw) - 1)) + k0f * L.ks;
    const uint64_t pol = adj_policy_evict_first();

    auto fetch = [&](int g) {
        if (g < ngroups && okf) {
            const int j0 = g * GS;
            const int cnt = min(GS, nwin - j0);
            float2 *dst = ring + (size_t)(g % NS) * GS * slot + sdst;
            const float2 *src = gsrc + (int64_t)(qb - 1 - j0) * grow;
            for (int st = 0; st < cnt; ++st) {
                if (q16) {
                    constexpr int KS = 2 * R;  // 128 threads over CH / 2 pairs
                    if constexpr (n >= KS) {
#pragma unroll
                        for (int t = 0; t < n / KS; ++t)
                            adj_cp_async_16_hint(dst + t * KS * L.ks, src + t * KS * n1, pol);
                    } else {
                        adj_cp_async_16_hint(dst, src, pol);  // k0f < n
                    }
                } else {
                    for (int t = 0; k0f + R * t < n; ++t) adj_cp_async_8(dst + t * R * L.ks, src + t * R * n1, true, pol);
                }
                dst += slot;
                src -= grow;
            }
        }
        adj_cp_async_commit();  // one group per stage, empty past the last
    };
#pragma unroll
    for (int g = 0; g < NS - 1; ++g) fetch(g);

    // this thread's word within a staged step, and the stride between its k0 values
    const int tbase = (chl >> L.lw) * L.gs + (chl & ((1 << L.lw) - 1)) + c * L.ks;
    const int tstride = R * L.ks;
    float2 *gz = p.gz[blockIdx.z];
    float2 *side = p.side[blockIdx.z] + (int64_t)blockIdx.y * (n - 1) * p.nch + ch;

    Tree tree;
    tree.init(c, p.om64);
    for (int jb = 0; jb < steps; jb += UNR) {
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            const int g = j / GS;
            if constexpr (J % GS == 0) {
                if (j < steps) {
                    adj_cp_async_wait_n<NS - 2>();  // this thread's copies of stage g are done
                    __syncthreads();  // everyone's are visible; the slot of stage g - 1 is free
                    fetch(g + NS - 1);
                }
            }
            if (j < steps) {
                const int r = p_hi - j;  // z row (window end row) of this step
                float2 y;
                if (kTail && j >= nwin + n / 2 - 1) {
                    // the last n/2 rows: no window of the chunk reaches them through level 1
                    if constexpr (kTail) y = tree.template tail<J>();
                } else {
                    float2 u[Tree::kIn];
                    if (j < nwin) {
                        const float2 *src = ring + ((size_t)(g % NS) * GS + (J % GS)) * slot + tbase;
#pragma unroll
                        for (int t = 0; t < Tree::kIn; ++t) u[t] = src[t * tstride];
                    } else {
#pragma unroll
                        for (int t = 0; t < Tree::kIn; ++t) u[t] = make_float2(0.f, 0.f);
                    }
                    y = tree.template step<J>(u);
                }
#pragma unroll
                for (int off = CPW; off < 32; off <<= 1) {  // the residues of one channel
                    y.x += __shfl_xor_sync(0xffffffffu, y.x, off);
                    y.y += __shfl_xor_sync(0xffffffffu, y.y, off);
                }
                y = c_scale(s, y);
                if (c == 0 && active) {
                    if (r >= qb && !last)
                        side[(int64_t)(r - qb) * p.nch] = y;
                    else
                        gz[(int64_t)r * p.nch + ch] = y;
                }
            }
        });
    }
    adj_cp_async_wait_0();  // (every stage was consumed above; nothing is left in flight)
}

// gz staging for adj_row: a block's rows (128 >> B of them) need n1 values per row per step,
// consecutive steps reading consecutive (descending) q1, so GS steps of one row are one
// contiguous run of GS * n1 values.  Groups of GS steps (16 KB per block) are copied by
// cp.async into a double-buffered ring, one group ahead of use, 16 bytes per copy (8 for
// n1 = 1); rows are padded by R values so that the 2^B lanes of 32 / 2^B rows hit distinct banks.
template <int M, int B>
struct AdjRowStage {
    static constexpr int R = 1 << B;
    static constexpr int kRows = 128 >> B;  // rows per block
    static constexpr int kN = 1 << M;
    static constexpr int kGS0 = 2048 / (kRows * kN);
    static constexpr int kGS = kGS0 < 1 ? 1 : (kGS0 > 16 ? 16 : kGS0);  // steps per group
    static constexpr int kRow = kGS * kN + R;    // staged values per row (padded)
    static constexpr int kPiece = kN >= 2 ? 2 : 1;  // values per copy
    static constexpr int kPerRow = kGS * kN / kPiece;  // copies per row per group
    static constexpr size_t kBytes = sizeof(float2) * 2 * kRows * kRow;
    static_assert(kPerRow <= 128 && 128 % kPerRow == 0, "copies of a group must tile the block");
    static_assert(kPiece == 1 || kRow % 2 == 0, "16-byte copies need 16-byte aligned rows");
};

template <int M, int B>
__host__ __device__ constexpr size_t adj_row_smem() { return AdjRowStage<M, B>::kBytes; }

__device__ __forceinline__ void adj_cp_async_16(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void adj_cp_async_8_plain(void *smem, const void *gmem, bool valid) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}

template <int M, int B, bool CPLX>
__global__ void __launch_bounds__(128) adj_row_kernel(const __grid_constant__ AdjRowParams p) {
    using Tree = SlidingTreeAdjoint<M, B>;
    using St = AdjRowStage<M, B>;
    constexpr int R = St::R;
    constexpr int n = St::kN;
    constexpr int GS = St::kGS;
    constexpr int UNR = Tree::kPeriod > GS ? Tree::kPeriod : GS;
    extern __shared__ float2 sz[];  // [2][kRows][kRow]

    const int c = threadIdx.x & (R - 1);
    const int rl = threadIdx.x >> B;  // this thread's row within the block
    const int row0 = blockIdx.x * St::kRows;
    const int row = row0 + rl;
    const bool active = row < p.zrows;
    const int pa = blockIdx.y * p.chunk;
    if (pa >= p.N1) return;  // uniform per block
    const int pb = min(pa + p.chunk, p.N1);
    const int p_hi = min(pb + n - 2, p.N1 - 1);
    const int steps = p_hi - pa + 1;
    const int q1_top = p_hi - (n - 1);  // q1 of step 0; step j reads q1_top - j

    const int64_t rowlen = (int64_t)p.P1 * n;
    const float2 *gz = p.gz[blockIdx.z];
    void *gx = p.gx[blockIdx.z];

    // copying thread i always takes piece i mod kPerRow of rows i / kPerRow + t * (128 / kPerRow)
    constexpr int kRowStep = 128 / St::kPerRow;
    constexpr int kCopies = St::kRows / kRowStep;
    const int off_f = (threadIdx.x % St::kPerRow) * St::kPiece;  // value offset in the group's run
    const int rl_f = threadIdx.x / St::kPerRow;
    const int dq_f = off_f / n;  // q1 of this piece relative to the group's lowest q1
    auto fetch = [&](int j0, int b) {
        const int q1lo = q1_top - j0 - (GS - 1);
        const int q = q1lo + dq_f;
        const bool qok = q >= 0 && q < p.P1;
        const int64_t goff = (int64_t)q1lo * n + off_f;
        float2 *dst = sz + (b * St::kRows + rl_f) * St::kRow + off_f;
#pragma unroll
        for (int t = 0; t < kCopies; ++t) {
            const int r = row0 + rl_f + t * kRowStep;
            const bool ok = qok && r < p.zrows;
            const float2 *src = ok ? gz + (int64_t)r * rowlen + goff : gz;
            if constexpr (St::kPiece == 2)
                adj_cp_async_16(dst + t * kRowStep * St::kRow, src, ok);
            else
                adj_cp_async_8_plain(dst + t * kRowStep * St::kRow, src, ok);
        }
        adj_cp_async_commit();
    };

    Tree tree;
    tree.init(c, p.om64);
    fetch(0, 0);
    for (int jb = 0; jb < steps; jb += UNR) {
        static_for<0, UNR>([&](auto JJ) {
            constexpr int J = decltype(JJ)::value;
            const int j = jb + J;
            if constexpr (J % GS == 0) {
                if (j + GS < steps) {
                    fetch(j + GS, ((j / GS) + 1) & 1);
                    adj_cp_async_wait_1();
                } else {
                    adj_cp_async_wait_0();
                }
                __syncthreads();
            }
            if (j < steps) {
                const int p1 = p_hi - j;
                const float2 *src = sz + (((j / GS) & 1) * St::kRows + rl) * St::kRow + (GS - 1 - (J % GS)) * n + c;
                float2 u[Tree::kIn];
#pragma unroll
                for (int t = 0; t < Tree::kIn; ++t) u[t] = src[t * R];
                const float2 y = reduce_residues<R>(tree.template step<J>(u));
                if (c == 0 && active && p1 < pb) {
                    if constexpr (CPLX)
                        reinterpret_cast<float2 *>(gx)[(int64_t)row * p.ld_out + p1] = y;
                    else
                        reinterpret_cast<float *>(gx)[(int64_t)row * p.ld_out + p1] = y.x;
                }
            }
            if constexpr (J % GS == GS - 1) __syncthreads();  // the buffer is refilled next group
        });
    }
}

template <int M, int B>
void adj_col_ring_launch_mb(const AdjColRingParams &p, dim3 g, dim3 b, size_t smem, cudaStream_t s);
template <int M, int B>
void adj_row_launch_mb(const AdjRowParams &p, int cplx, dim3 g, dim3 b, cudaStream_t s);
template <int M, int B>
int adj_row_bps_mb(int cplx);  // resident 128-thread blocks per SM (occupancy API; 0 on error)

// The residue split each adjoint pass uses for a window side 2^M (registers without spills).
__host__ __device__ constexpr int adj_col_B(int M) { return M <= 4 ? (M < 1 ? M : 1) : M - 3; }
__host__ __device__ constexpr int adj_row_B(int M) { return M >= 4 ? 3 : (M < 2 ? M : 2); }

#define SWDFT_ADJ_INSTANTIATE(M_)                                                                 \
    template <>                                                                                  \
    void adj_row_launch_mb<M_, adj_row_B(M_)>(const AdjRowParams &p, int cplx, dim3 g, dim3 b,   \
                                              cudaStream_t s) {                                  \
        constexpr size_t smem = adj_row_smem<M_, adj_row_B(M_)>();                               \
        static const bool attr_set =                                                             \
            smem <= 48 * 1024 ||                                                                 \
            (cudaFuncSetAttribute(adj_row_kernel<M_, adj_row_B(M_), true>,                       \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==     \
                 cudaSuccess &&                                                                  \
             cudaFuncSetAttribute(adj_row_kernel<M_, adj_row_B(M_), false>,                      \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==     \
                 cudaSuccess);                                                                   \
        (void)attr_set;                                                                          \
        if (cplx)                                                                                \
            adj_row_kernel<M_, adj_row_B(M_), true><<<g, b, smem, s>>>(p);                       \
        else                                                                                     \
            adj_row_kernel<M_, adj_row_B(M_), false><<<g, b, smem, s>>>(p);                      \
    }                                                                                            \
    template <>                                                                                  \
    int adj_row_bps_mb<M_, adj_row_B(M_)>(int cplx) {                                            \
        constexpr size_t smem = adj_row_smem<M_, adj_row_B(M_)>();                               \
        int nb = 0;                                                                              \
        cudaError_t e = cplx ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                                   &nb, adj_row_kernel<M_, adj_row_B(M_), true>, 128, smem)      \
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                                   &nb, adj_row_kernel<M_, adj_row_B(M_), false>, 128, smem);    \
        return e == cudaSuccess ? nb : 0;                                                        \
    }

// The ring-staged adj_col for window side 2^M_: launch (dynamic shared memory set once to the
// largest layout of any n1).
#define SWDFT_ADJ_RING_INSTANTIATE(M_)                                                            \
    template <>                                                                                  \
    void adj_col_ring_launch_mb<M_, adj_col_B(M_)>(const AdjColRingParams &p, dim3 g, dim3 b,    \
                                                   size_t smem, cudaStream_t s) {                \
        static const bool attr_set = [] {                                                        \
            size_t mx = 0;                                                                       \
            for (int m1 = 0; m1 <= kMaxLog2; ++m1)                                               \
                mx = std::max(mx, adj_col_smem(M_, adj_col_layout(M_, adj_col_B(M_), m1).slot)); \
            return cudaFuncSetAttribute(adj_col_ring_kernel<M_, adj_col_B(M_)>,                  \
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx) == \
                   cudaSuccess;                                                                  \
        }();                                                                                     \
        (void)attr_set;                                                                          \
        adj_col_ring_kernel<M_, adj_col_B(M_)><<<g, b, smem, s>>>(p);                            \
    }

}  // namespace swdft
