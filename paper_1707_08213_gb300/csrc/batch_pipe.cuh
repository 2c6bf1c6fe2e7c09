// Pipelined persistent launch over the two-pass arrays of a batch that share a window shape
// (n0, n1) = (2^M0, 2^M1): one kernel evaluates both passes.
//
// Work is a list of tiles in ticket order, built on the host (build_pipe): row tiles (Eq.
// rowfswft2d, `row_tile`: a block of z rows x a chunk of window columns) interleaved with the
// column tiles (Eq. colfswft2d, `col_tile`: 32 channels x a chunk of window rows) that read
// them, each column tile placed at least a full set of resident blocks after its row tiles
// (with a cap on the z written ahead).  A block takes the next ticket from a counter
// (fetched one tile ahead), so tiles start in list order whatever the residency.  A finished
// row tile raises its flag (one per (array, row block, row chunk); release at GPU scope); a
// column tile first waits until the flags of every row tile it reads from are up -- the lanes
// of warp 0 poll them in parallel, then acquire.  Every wait is on an earlier ticket, and the
// earliest unfinished ticket is always running (row tiles never wait), so the launch cannot
// deadlock; each wait is still bounded by a clock64 budget, after which the lane records the
// time-out (this unit's status word and the launch's abort word) and every block of the
// launch stops at its next tile.  z of a row block is read a few tiles after it is written,
// from L2.
#pragma once

#include "batch_fused.cuh"
#include "tree_kernels.cuh"

namespace swdft {

// Row tiles inside the pipelined kernel: 2^B residue threads per z row.  n1 = 64 takes B = 3
// (8 outputs per thread) so the row tree fits the column tile's register budget.
__host__ __device__ constexpr int bpipe_row_B(int m1) { return m1 >= 5 ? 3 : (m1 < 3 ? m1 : 3); }
__host__ __device__ constexpr int bpipe_rows_per_tile(int m0, int m1) { return bfu_threads(m0) >> bpipe_row_B(m1); }
// Resident blocks: the column tile's bound, lowered where the row tree needs more registers
// (n1 = 32, 64) so that neither spills beyond a few words.
__host__ __device__ constexpr int bpipe_min_blocks(int m0, int m1) {
    return m1 >= 6 ? (m0 >= 6 ? 1 : 3) : (m1 == 5 && bcol_min_blocks(m0) > 6 ? 6 : bcol_min_blocks(m0));
}

struct BatchPipeParams {
    const BatchImage *imgs;
    const BatchPipeItem *items;  // this class's tiles in ticket order
    int *ticket;                 // next ticket of this launch (zeroed before the launch)
    int *abort;                  // nonzero once a wait gave up: every block stops
    int *done;                   // per (array, row block, row chunk): 1 once the row tile finished
    int nitems;
    int poison;                  // test hook: added to the flag value array 0's column tiles wait for
    long long budget;            // clock64 cycles one column tile may wait
    Omega64 om;
};

__device__ __forceinline__ int pipe_ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void pipe_red_release(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// with a preceding relaxed load that saw the flag, an acquire (orders this thread's later
// loads after it without waiting for its earlier stores)
__device__ __forceinline__ void pipe_fence_acquire() { asm volatile("fence.acquire.gpu;" ::: "memory"); }

static __device__ int g_pipe_status;  // one word per translation unit: a wait gave up

template <int M0, int M1>
__global__ void __launch_bounds__(bfu_threads(M0), bpipe_min_blocks(M0, M1))
    batch_pipe_kernel(const __grid_constant__ BatchPipeParams p) {
    extern __shared__ float2 ring[];
    __shared__ int s_ticket;
    __shared__ int s_go;
    constexpr int n0 = 1 << M0;
    constexpr int RB1 = bpipe_row_B(M1);
    constexpr int rpb = bpipe_rows_per_tile(M0, M1);
    const int lane = threadIdx.x & 31;
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(p.ticket, 1);
    for (;;) {
        if (threadIdx.x == 0) {
            s_ticket = *(volatile int *)p.abort ? p.nitems : next;
            if (s_ticket < p.nitems) next = atomicAdd(p.ticket, 1);  // the following tile's ticket, in flight
        }
        __syncthreads();
        const int t = s_ticket;
        if (t >= p.nitems) return;  // uniform
        const BatchPipeItem it = p.items[t];
        const BatchImage &d = p.imgs[it.img];
        if (it.code >= 0) {
            const int rb = it.code / d.row_chunks;
            const int rc = it.code - rb * d.row_chunks;
            if (d.cplx)
                row_tile<M1, RB1, true>(d.row, rb, rc, p.om.w);
            else
                row_tile<M1, RB1, false>(d.row, rb, rc, p.om.w);
            __syncthreads();  // every thread's z stores precede the release below
            if (threadIdx.x == 0) pipe_red_release(p.done + d.sync_off + it.code, 1);
            continue;
        }
        const int code = ~it.code;
        const int ck = code / d.col_blocks;
        const int cb = code - ck * d.col_blocks;
        if (threadIdx.x < 32) {
            // the row tiles of z rows [r_lo, r_hi) and of this tile's window columns
            int r_lo, r_hi;
            pipe_col_rows(ck, d.col.chunk, d.col.rows_out, n0, &r_lo, &r_hi);
            const int rb_lo = r_lo / rpb, nrb = (r_hi - 1) / rpb - rb_lo + 1;
            const int64_t ch_lo = (int64_t)cb * 32 * d.col.groups;
            const int64_t ch_end = ch_lo + 32 * d.col.groups;
            const int64_t ch_hi = (ch_end < d.col.nch ? ch_end : d.col.nch) - 1;
            const int rc_lo = (int)((ch_lo >> d.col.m1) / d.row.chunk);
            const int nrc = (int)((ch_hi >> d.col.m1) / d.row.chunk) - rc_lo + 1;
            const int need = 1 + (it.img == 0 ? p.poison : 0);
            int go = 1;
            const long long t0 = clock64();
            for (int f = lane; f < nrb * nrc && go; f += 32) {
                const int rb = rb_lo + f / nrc, rc = rc_lo + f % nrc;
                const int *flag = p.done + d.sync_off + rb * d.row_chunks + rc;
                while (pipe_ld_relaxed(flag) < need) {
                    if (*(volatile int *)p.abort) {
                        go = 0;
                        break;
                    }
                    if (clock64() - t0 > p.budget) {
                        atomicExch(p.abort, 1);
                        atomicExch(&g_pipe_status, 1);
                        go = 0;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            pipe_fence_acquire();  // the row tiles' z stores are visible from here on
            go = __all_sync(0xffffffffu, go);
            if (lane == 0) s_go = go;
        }
        __syncthreads();
        if (!s_go) return;  // uniform: the launch is stopping
        col_tile<M0, bfu_B(M0)>(d.col, cb, ck, p.om.w, ring);  // ends with a barrier
    }
}

// launcher, occupancy and status word for one M0 (all m1), defined in batch_pipe_m*.cu
template <int M0>
cudaError_t bpipe_launch(int m1, const BatchPipeParams &p, unsigned grid, cudaStream_t s);
template <int M0>
cudaError_t bpipe_bps(int m1, int *bps);
template <int M0>
cudaError_t bpipe_status_mb(int *status, bool reset);

#define SWDFT_BPIPE_CASES(M0_, X) X(M0_, 0) X(M0_, 1) X(M0_, 2) X(M0_, 3) X(M0_, 4) X(M0_, 5) X(M0_, 6)

#define SWDFT_BPIPE_INSTANTIATE(M0_)                                                                   \
    template <>                                                                                        \
    cudaError_t bpipe_launch<M0_>(int m1, const BatchPipeParams &p, unsigned grid, cudaStream_t s) {   \
        const size_t smem = bfu_smem(M0_);                                                             \
        switch (m1) {                                                                                  \
            SWDFT_BPIPE_CASES(M0_, SWDFT_BPIPE_LAUNCH_CASE)                                            \
            default: return cudaErrorInvalidValue;                                                     \
        }                                                                                              \
        return cudaGetLastError();                                                                     \
    }                                                                                                  \
    template <>                                                                                        \
    cudaError_t bpipe_bps<M0_>(int m1, int *bps) {                                                     \
        const size_t smem = bfu_smem(M0_);                                                             \
        switch (m1) {                                                                                  \
            SWDFT_BPIPE_CASES(M0_, SWDFT_BPIPE_BPS_CASE)                                               \
            default: return cudaErrorInvalidValue;                                                     \
        }                                                                                              \
    }                                                                                                  \
    template <>                                                                                        \
    cudaError_t bpipe_status_mb<M0_>(int *status, bool reset) {                                        \
        cudaError_t e = cudaMemcpyFromSymbol(status, g_pipe_status, sizeof(int));                      \
        if (e == cudaSuccess && reset && *status != 0) {                                               \
            const int zero = 0;                                                                        \
            e = cudaMemcpyToSymbol(g_pipe_status, &zero, sizeof(int));                                 \
        }                                                                                              \
        return e;                                                                                      \
    }

#define SWDFT_BPIPE_LAUNCH_CASE(M0_, M1_)                                                  \
    case M1_:                                                                              \
        batch_pipe_kernel<M0_, M1_><<<grid, bfu_threads(M0_), smem, s>>>(p);               \
        break;
#define SWDFT_BPIPE_BPS_CASE(M0_, M1_)                                                     \
    case M1_:                                                                              \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_pipe_kernel<M0_, M1_>, \
                                                             bfu_threads(M0_), smem);

}  // namespace swdft
