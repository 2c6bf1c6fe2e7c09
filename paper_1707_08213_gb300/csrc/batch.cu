// Persistent launches over a batch of arrays of uneven sizes and window shapes (host side).
//
// Arrays whose window has n0 n1 <= 64 run in fused groups, one persistent kernel per (n0, n1)
// (batch_fused.cuh): column tiles that evaluate their own row levels, no z.  Every other array
// runs in the pipelined kernel of its (n0, n1) (batch_pipe.cuh): row tiles and the column
// tiles that read them in one launch, ordered per array so that z is consumed from L2.  The
// kernels of a batch run concurrently on the plan's side streams; each has a grid of SMs x
// resident blocks, and a block finds its tile's array from the tile (by a ticket into the
// item table for the pipelined kernels, by binary search over the group's tile offsets for
// the fused ones) and calls the same tile functions the per-array kernels use.  Every array
// has its own z region of the workspace.
#include <algorithm>

#include "batch_fused.cuh"
#include "batch_pipe.cuh"
#include "tree_kernels.cuh"

namespace swdft {

// Launch choices of the fused groups' column tiles for a window side of 2^m: 128 threads (256
// for 64-point trees; bfu_B / bfu_threads / bfu_groups of batch_fused.cuh).
static_assert(32 * (1 << bfu_B(6)) * bfu_groups(6) == bfu_threads(6) &&
                  32 * (1 << bfu_B(5)) * bfu_groups(5) == bfu_threads(5),
              "column tiles: 2^B residue warps x 32-channel groups fill the block");

int batch_col_B(int m0) { return bfu_B(m0); }
int batch_col_groups(int m0) { return bfu_groups(m0); }

cudaError_t batch_fused_blocks_per_sm(int m0, int m1, int *bps) {
    if (m1 < 0 || m1 >= kBatchFusedM1) return cudaErrorInvalidValue;
    switch (m0) {
        case 0: return bfu_bps<0>(m1, bps);
        case 1: return bfu_bps<1>(m1, bps);
        case 2: return bfu_bps<2>(m1, bps);
        case 3: return bfu_bps<3>(m1, bps);
        case 4: return bfu_bps<4>(m1, bps);
        case 5: return bfu_bps<5>(m1, bps);
        case 6: return bfu_bps<6>(m1, bps);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_fused_class(int m0, int m1, const BatchImage *d_images, const BatchClassEntry *ent,
                                     int nent, int64_t nitems, const float2 *om64, int64_t slots, cudaStream_t s) {
    if (nent <= 0 || nitems <= 0) return cudaSuccess;
    Omega64 om;
    for (int j = 0; j < kMaxN; ++j) om.w[j] = om64[j];
    const unsigned grid = (unsigned)std::min<int64_t>(nitems, std::max<int64_t>(1, slots));
    switch (m0) {
        case 0: return bfu_launch<0>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 1: return bfu_launch<1>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 2: return bfu_launch<2>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 3: return bfu_launch<3>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 4: return bfu_launch<4>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 5: return bfu_launch<5>(m1, d_images, ent, nent, nitems, om, grid, s);
        case 6: return bfu_launch<6>(m1, d_images, ent, nent, nitems, om, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int batch_pipe_rows_per_tile(int m0, int m1) { return bpipe_rows_per_tile(m0, m1); }
int batch_pipe_row_B(int m1) { return bpipe_row_B(m1); }

cudaError_t batch_pipe_blocks_per_sm(int m0, int m1, int *bps) {
    if (m1 < 0 || m1 > kMaxLog2) return cudaErrorInvalidValue;
    switch (m0) {
        case 0: return bpipe_bps<0>(m1, bps);
        case 1: return bpipe_bps<1>(m1, bps);
        case 2: return bpipe_bps<2>(m1, bps);
        case 3: return bpipe_bps<3>(m1, bps);
        case 4: return bpipe_bps<4>(m1, bps);
        case 5: return bpipe_bps<5>(m1, bps);
        case 6: return bpipe_bps<6>(m1, bps);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t batch_pipe_status(int *status, bool reset) {
    *status = 0;
    for (int m0 = 0; m0 <= kMaxLog2; ++m0) {
        int st = 0;
        cudaError_t e = cudaSuccess;
        switch (m0) {
            case 0: e = bpipe_status_mb<0>(&st, reset); break;
            case 1: e = bpipe_status_mb<1>(&st, reset); break;
            case 2: e = bpipe_status_mb<2>(&st, reset); break;
            case 3: e = bpipe_status_mb<3>(&st, reset); break;
            case 4: e = bpipe_status_mb<4>(&st, reset); break;
            case 5: e = bpipe_status_mb<5>(&st, reset); break;
            case 6: e = bpipe_status_mb<6>(&st, reset); break;
        }
        if (e != cudaSuccess) return e;
        if (st) *status = 1;
    }
    return cudaSuccess;
}

cudaError_t launch_batch_pipe(int m0, int m1, const BatchPipeArgs &a, int64_t slots, cudaStream_t s) {
    if (a.nitems <= 0) return cudaSuccess;
    if (m1 < 0 || m1 > kMaxLog2 || !a.imgs || !a.items || !a.ticket || !a.abort || !a.done || !a.om64)
        return cudaErrorInvalidValue;
    BatchPipeParams p;
    p.imgs = a.imgs;
    p.items = a.items;
    p.ticket = a.ticket;
    p.abort = a.abort;
    p.done = a.done;
    p.nitems = a.nitems;
    p.poison = a.poison;
    p.budget = a.budget;
    for (int j = 0; j < kMaxN; ++j) p.om.w[j] = a.om64[j];
    const unsigned grid = (unsigned)std::min<int64_t>(a.nitems, std::max<int64_t>(1, slots));
    switch (m0) {
        case 0: return bpipe_launch<0>(m1, p, grid, s);
        case 1: return bpipe_launch<1>(m1, p, grid, s);
        case 2: return bpipe_launch<2>(m1, p, grid, s);
        case 3: return bpipe_launch<3>(m1, p, grid, s);
        case 4: return bpipe_launch<4>(m1, p, grid, s);
        case 5: return bpipe_launch<5>(m1, p, grid, s);
        case 6: return bpipe_launch<6>(m1, p, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swdft
