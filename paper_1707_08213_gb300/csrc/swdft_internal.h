// Internal interfaces between the C-ABI host code (api.cpp) and the kernel translation
// units.  Nothing here is exported.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace swdft {

// Fault injection (swdft2d_inject_alloc_failure): true when the allocation about to be made
// must fail.  Every allocation the library makes asks first, host and device alike.
bool alloc_fails();


// Tree kernels keep every butterfly level of one window axis in registers; they are built
// for window lengths up to 2^kMaxLog2 along each axis.
constexpr int kMaxLog2 = 6;
constexpr int kMaxN = 1 << kMaxLog2;
// Ternary and mixed-radix trees (tree3.cu) are built for window lengths 3^b 2^a <= 64 with
// 1 <= b <= kMaxLog3.
constexpr int kMaxLog3 = 3;
constexpr int kMaxN3 = 27;

// Omega^i of Section 4.2 for length n (any n >= 1), FP64-evaluated, FP32-rounded.
void make_omega(int n, float2 *out);

// Default launch shapes of the binary tree's two passes over a band of window rows (used by
// the plans and by the allocation-free entry point alike; measured on the 512x512/32x32 and
// 1024x2048/16x64 workloads).
//  * row levels: thread = (row, residue, chunk of window columns); B = 3 (2 for 64-point
//    trees, which need more registers), about 64K threads in flight, chunks no shorter than
//    n1/2 (each chunk's walk starts n1/2 columns before its first window: n1/2 - 1 steps of
//    warm-up).
//  * column levels: thread = (channel, residue, chunk of window rows); B = 2 (3 for 64-point
//    trees); about eight row chunks per 32-channel group (sixteen for fused small windows;
//    the plans give the fused form of larger windows two),
//    more when there are few channel groups, so that the pass has at least four blocks per
//    SM; every chunk at least 2 n0 rows (its walk has n0/2 - 1 steps of warm-up; n0 - 1 for
//    TMA-staged walks of n0 <= 8, which start on a whole step group of 8 rows).
inline int default_row_B(int m1) { return m1 >= 6 ? 2 : (m1 < 3 ? m1 : 3); }
inline int64_t default_row_chunk(int64_t P1, int64_t zrows, int64_t threads_per_row, int n1) {
    const int64_t t = zrows * threads_per_row;
    const int64_t nchunk = (64LL << 10) / (t > 1 ? t : 1);
    const int64_t nc = nchunk > 1 ? nchunk : 1;
    const int64_t chunk = (P1 + nc - 1) / nc;
    const int64_t lo = n1 / 2 > 1 ? n1 / 2 : 1;
    const int64_t c = chunk > lo ? chunk : lo;
    return c < P1 ? c : P1;
}
inline int default_col_B(int m0) { return m0 >= 6 ? 3 : (m0 < 2 ? m0 : 2); }
inline int default_col_nchunks(int64_t nch, int sm_count, bool fused_small) {
    const int64_t ch_groups = (nch + 31) / 32;
    const int64_t want = (4LL * (sm_count > 1 ? sm_count : 1) + ch_groups - 1) / ch_groups;
    const int64_t base = fused_small ? 16 : 8;
    const int64_t n = want > base ? want : base;
    return (int)(n < 65535 ? n : 65535);
}
inline int64_t default_col_chunk(int64_t band_rows, int n0, int nchunks) {
    const int64_t chunk = (band_rows + nchunks - 1) / nchunks;
    const int64_t c = chunk > 2LL * n0 ? chunk : 2LL * n0;
    return c < band_rows ? c : band_rows;
}

// Geometry of one row-level pass (see RowTreeArgs): z[r][q1][k1] for `rows` input rows.
struct RowGeom {
    const void *x;
    int64_t ld;       // input row stride, elements
    int64_t r_base;   // first input row
    int64_t zrow;     // elements per z row (P1 * n1)
    int rows;
    int P1;
    int chunk;        // window columns per thread
    float2 *z;        // first (non-padding) z row
};

// Geometry of one column-level pass (see ColTreeArgs).
struct ColGeom {
    const float2 *z;  // first (non-padding) z row
    float2 *out;
    int64_t nch;      // channels = P1 * n1 = elements per z row
    int64_t orow;     // elements per output row = P1 * n0 * n1
    int rows_out;
    int chunk;        // window rows per thread
    int m1;           // log2 of the coefficients per window column (n1; prod n_e in kD)
    int groups;       // 32-channel groups per block
    float scale;
    int64_t zslice;   // elements between slices of z / of the output (grid z, kD passes)
    int64_t oslice;
};

// One array of a persistent batch launch: its geometry and how its row and column passes
// are cut into block tiles (row tiles = row_blocks x row_chunks, column tiles likewise).
struct BatchImage {
    RowGeom row;
    ColGeom col;
    int m0, m1, cplx;
    int fused;  // row levels inside the column tile (no row tiles, no z)
    int row_blocks, row_chunks;  // row pass: blocks of (128 >> B) rows x chunks of columns
    int col_blocks, col_chunks;  // column pass: blocks of 32 * groups channels x row chunks
    int sync_off;                // pipelined launch: first of this array's row-tile flags
    int pad_;
};

// Tensor-core column levels: out[q0][q1][k0][k1] = scale * sum_j0 z[q0+j0][ch] F0[j0][k0]
// from 16-bit operand planes of z ([plane][rows_out + n0 - 1][P1*n1]; planes Re hi, Im hi,
// Re lo, Im lo for terms = 3, Re, Im for terms = 1).  16 <= n0 <= 64, 8 <= n1 <= 64.
struct TcColArgs {
    void *planes = nullptr;
    int terms = 3;
    bool f16 = false;
    const float *amax = nullptr;  // per-image fp16 scaling: amax * amax_mult bounds |z|
    float amax_mult = 1.f;
    int64_t P1 = 0, rows_out = 0;
    int m0 = 0, m1 = 0;
    float2 *out = nullptr;
    float scale = 1.f;
    const float2 *om64 = nullptr;
    int64_t chunk = 0;  // window rows per CTA
};
cudaError_t launch_tc_col(const TcColArgs &a, cudaStream_t s);
size_t tc_col_smem_bytes(int m0, int terms, int chunk);

// Tensor-core row levels: writes z[r][q1][k1] = sum_j1 x[r][q1+j1] F1[j1][k1] for the band's
// zrows input rows directly as the column pass's operand planes.  With amax (fp16 forms with
// the per-image scale) the kernel first stores max |x| there and scales by the power of two
// that fits n1 * max|x| below 2^14.
struct TcRowArgs {
    const void *x = nullptr;  // first input row of the band
    int64_t ld = 0;
    int cplx = 0;
    int64_t N1 = 0, P1 = 0, zrows = 0;
    int m1 = 0;
    void *planes = nullptr;
    int terms = 3;
    bool f16 = false;
    float *amax = nullptr;
    const float2 *om64 = nullptr;
};
cudaError_t launch_tc_row(const TcRowArgs &a, cudaStream_t s);
// Device error word of the tensor-core kernels (1 = a bounded wait timed out).
cudaError_t tc_status(int *status, bool reset);
// One block whose bounded mbarrier wait runs out on purpose (selftest.cu; no fault), and its
// own device word (1 = that wait timed out).
cudaError_t launch_wait_timeout_probe(uint32_t polls, cudaStream_t s);
cudaError_t probe_status(int *status, bool reset);

// One array of a window-exponent group in a persistent batch launch: item0 = the group's
// first tile of this array (tiles are numbered array by array within the group).
struct BatchClassEntry {
    int64_t item0;
    int img;
    int pad;
};
// Fused groups (arrays with n0 = 2^m0, n1 = 2^m1, m1 <= 5): column tiles that evaluate their
// own row levels from the input, as fused_tree_kernel does for one array.
constexpr int kBatchFusedM1 = 6;  // m1 = 0..5
cudaError_t launch_batch_fused_class(int m0, int m1, const BatchImage *d_images, const BatchClassEntry *ent,
                                     int nent, int64_t nitems, const float2 *om64, int64_t slots, cudaStream_t s);
cudaError_t batch_fused_blocks_per_sm(int m0, int m1, int *bps);
// Pipelined launches (batch_pipe.cuh): one per (n0, n1) = (2^m0, 2^m1) of the two-pass
// arrays, both passes in one kernel.  Device pointers; the counters are zeroed before the
// launch.  grid = min(nitems, slots).
struct BatchPipeItem {
    int img;   // index into the image table
    int code;  // >= 0: row tile rb * row_chunks + rc; < 0: column tile ~(ck * col_blocks + cb)
};
// z rows [r_lo, r_hi) of the band that column chunk ck reads (its ring starts n0/2 rows before
// the chunk's first window row, the column tree's look-back; padding rows below 0 are never
// written and never waited for).
constexpr void pipe_col_rows(int ck, int chunk, int rows_out, int n0, int *r_lo, int *r_hi) {
    const int qa = ck * chunk;
    const int qb = qa + chunk < rows_out ? qa + chunk : rows_out;
    const int look = n0 >= 2 ? n0 / 2 : 0;
    *r_lo = qa - look > 0 ? qa - look : 0;
    *r_hi = qb + n0 - 1;
}
struct BatchPipeArgs {
    const BatchImage *imgs = nullptr;
    const BatchPipeItem *items = nullptr;  // the class's tiles in ticket order
    int *ticket = nullptr, *abort = nullptr;
    int *done = nullptr;        // per (array, row block, row chunk) flags
    int nitems = 0;
    int poison = 0;             // test hook (swdft2d_debug_batch_wait)
    long long budget = 0;       // clock64 cycles a column tile may wait
    const float2 *om64 = nullptr;
};
cudaError_t launch_batch_pipe(int m0, int m1, const BatchPipeArgs &a, int64_t slots, cudaStream_t s);
cudaError_t batch_pipe_blocks_per_sm(int m0, int m1, int *bps);
cudaError_t batch_pipe_status(int *status, bool reset);
// z rows per row tile of a pipelined launch, and the residue split of its row trees
int batch_pipe_rows_per_tile(int m0, int m1);
int batch_pipe_row_B(int m1);
// Launch choices the batch kernels use for a window side of 2^m.
int batch_col_B(int m0);
int batch_col_groups(int m0);

// Row levels (Eq. rowfswft2d) of `rows` input rows starting at input row r_base:
//   z[r][q1][k1] = sum_{j1<n1} x[r_base + r][q1 + j1] w_{n1}^{-j1 k1}   (unnormalised)
// z is row-major rows x P1 x n1 complex64.
struct RowTreeArgs {
    const void *x = nullptr;  // N0 x N1 input, row stride ld elements
    int64_t ld = 0;
    int cplx = 0;             // 0: float32 input, 1: complex64
    int64_t r_base = 0;
    int64_t rows = 0;
    int64_t P1 = 0;
    int m1 = 0;               // log2 n1
    float2 *z = nullptr;
    const float2 *om64 = nullptr;  // host table w_64^{-j}, 64 entries (copied into kernel parameters)
    int B = 0;                // log2 of the threads sharing one row's butterflies
    int64_t chunk = 0;        // output positions per thread (plus n1-1 warm-up steps)
};

// Column levels (Eq. colfswft2d) of z, scaled and stored as the final output:
//   out[q0][q1][k0][k1] = scale * sum_{j0<n0} z[q0 + j0][q1][k1] w_{n0}^{-j0 k0}
// The same pass serves each earlier dimension of a k-dimensional transform (Eq. kdfswft):
// there q1 runs over the window positions of all later dimensions, k1 over their
// coefficients (m1 = the sum of their log2 lengths), and `slices` independent stacks of
// z rows (the positions of all earlier dimensions) are processed by one launch.
struct ColTreeArgs {
    const float2 *z = nullptr;  // (rows_out + n0 - 1) x P1 x n1
    int64_t P1 = 0;
    int64_t rows_out = 0;
    int m0 = 0, m1 = 0;
    float2 *out = nullptr;      // rows_out x P1 x n0 x n1
    float scale = 1.f;
    const float2 *om64 = nullptr;  // host table w_64^{-j}, 64 entries
    int B = 0;
    int64_t chunk = 0;          // output rows per thread (plus n0-1 warm-up steps)
    int groups = 1;             // 32-channel groups per block (block = 32 * 2^B * groups)
    int64_t slices = 1;         // stacks of z rows; slice s reads z + s*z_slice and
    int64_t z_slice = 0;        // writes out + s*out_slice (elements).  Rows before a
    int64_t out_slice = 0;      // slice's first row must be readable (padding / previous slice).
    // Optional, one stack: z_full = z's first padding row (z = z_full + z_pad * P1 * n1).
    // Given and 16-byte aligned with P1 * n1 even, the tiles' z rows are loaded by TMA.
    const float2 *z_full = nullptr;
    int64_t z_pad = 0;
};
// Device word of the TMA-staged column kernels (1 = a bounded wait gave up).
cudaError_t col_tma_status(int *status, bool reset);
// Largest m1 a column pass accepts (coefficient blocks of up to 2^18 per window column).
constexpr int kMaxInnerLog2 = 18;

cudaError_t launch_row_tree(const RowTreeArgs &a, cudaStream_t s);
// Column-pass launch geometry: the B and groups a launch actually uses, and how many
// blocks of that shape fit on one SM (occupancy API; 0 on error).
int col_tree_clamp_B(int m0, int B);
int col_tree_clamp_groups(int m0, int B, int groups);
int col_tree_blocks_per_sm(int m0, int B, int groups);
cudaError_t launch_col_tree(const ColTreeArgs &a, cudaStream_t s);

// Fused tree, n1 <= 64: one kernel evaluates the row levels of each z row inside the column
// tile (a warp per 32 channels) and the column levels as col_tree does; z never reaches HBM.
struct FusedTreeArgs {
    const void *x = nullptr;  // first input row of the band
    int64_t ld = 0;
    int cplx = 0;
    int64_t P1 = 0, rows_out = 0;
    int m0 = 0, m1 = 0;
    float2 *out = nullptr;
    float scale = 1.f;
    const float2 *om64 = nullptr;
    int64_t chunk = 0;
    int groups = 1;
};
cudaError_t launch_fused_tree(const FusedTreeArgs &a, cudaStream_t s);
// Window shapes the fused form is built for: n1 <= 32, and n1 = 64 with n0 <= 32 (64 x 64
// windows would need more registers than the fused kernel's two resident blocks allow).
inline bool fused_supported(int m0, int m1) { return m1 >= 0 && (m1 <= 5 || (m1 == 6 && m0 <= 5)); }

// Adjoint of the column levels: gz[r][q1][k1] = scale * sum_{j0,k0} G[r-j0][q1][k0][k1] w_{n0}^{+j0 k0}
// for the rows_out + n0 - 1 z rows of a band (G holds rows_out window rows).
// Work is split by window rows: chunks of `chunk` windows (>= n0-1; the last may be shorter),
// each reading its rows of G once.  The n0-1 gz rows after a chunk (not the last) are written
// to side[chunk index]; a second launch adds them into gz, so gz is complete on return.
// Arrays of one shape may share a launch: array z of nz (< kAdjZ) uses G[z], gz[z], side[z].
constexpr int kAdjZ = 8;
struct AdjColArgs {
    const float2 *G[kAdjZ] = {};
    float2 *gz[kAdjZ] = {};
    float2 *side[kAdjZ] = {};  // adj_side_elems(...) complex64 each, or null when there is one chunk
    int nz = 1;
    int64_t P1 = 0, rows_out = 0;
    int m0 = 0, m1 = 0;
    float scale = 1.f;
    const float2 *om64 = nullptr;  // host table w_64^{-j}, 64 entries
    int B = 0;
    int64_t chunk = 0;  // window rows per thread (plus n0-1 drain steps)
};
// Window rows per adj_col chunk the launcher actually uses, and its side buffer size.
int64_t adj_col_chunk(int64_t rows_out, int m0, int64_t requested);
int64_t adj_side_elems(int64_t rows_out, int m0, int64_t P1, int m1, int64_t requested);
// Kernel launches launch_adj_col makes (2 when chunk boundaries share rows, else 1).
int adj_col_launches(int64_t rows_out, int m0, int64_t requested);

// Adjoint of the row levels: gx[r][p1] = sum_{j1,k1} gz[r][p1-j1][k1] w_{n1}^{+j1 k1}
// (real part stored for float32 inputs), for zrows rows of N1 columns.
struct AdjRowArgs {
    const float2 *gz[kAdjZ] = {};
    void *gx[kAdjZ] = {};
    int nz = 1;
    int64_t ld_out = 0;
    int cplx = 0;
    int64_t zrows = 0, N1 = 0;
    int m1 = 0;
    const float2 *om64 = nullptr;  // host table w_64^{-j}, 64 entries
    int B = 0;
    int64_t chunk = 0;  // output columns per thread (plus n1-1 warm-up steps); 0: one wave
    int sm_count = 152;  // for chunk = 0
};

// Adjoint passes for ternary and mixed-radix windows (adjoint3.cu): dense inverse DFTs of
// length n per window, overlap-added in gather form.  Column pass: gz[r][q1][k1] = scale *
// sum over the windows q0 covering row r of sum_k0 G[q0][q1][k0][k1] w_{n0}^{+(r-q0) k0}
// (gz: rows_out + n0 - 1 rows of P1 n1 complex64; zeroed by the launcher).  Row pass:
// gx[r][p1] = sum over the windows q1 covering column p1 of sum_k1 gz[r][q1][k1]
// w_{n1}^{+(p1-q1) k1}, real part for float32 gradients (gx: zrows x N1, zeroed by the
// launcher).  n0: 1 or 3^b 2^a (b >= 1) <= 64; n1: 3^b 2^a (b >= 1) <= 64.
struct Adj3ColArgs {
    const float2 *G = nullptr;
    float2 *gz = nullptr;
    int64_t P1 = 0, rows_out = 0;
    int n0 = 1, n1 = 1;
    float scale = 1.f;
};
struct Adj3RowArgs {
    const float2 *gz = nullptr;
    void *gx = nullptr;
    int64_t ld_out = 0, zrows = 0, N1 = 0;
    int n1 = 1;
    int cplx = 0;
};
cudaError_t launch_adj3_col(const Adj3ColArgs &a, cudaStream_t s);
cudaError_t launch_adj3_row(const Adj3RowArgs &a, cudaStream_t s);

// Ternary and mixed-radix trees (tree3.cu): windows of n = 3^b 2^a samples along an axis
// (b >= 1, n <= 64; b = a = 0: one sample), radix-3 levels first.
// Row levels: z[r][q1][k1] for `rows` input rows (n1 = 3^b1 2^a1), as RowTreeArgs.
struct Row3Args {
    const void *x = nullptr;
    int64_t ld = 0;
    int cplx = 0;
    int64_t r_base = 0, rows = 0, P1 = 0;
    int b1 = 0, a1 = 0;             // n1 = 3^b1 2^a1
    float2 *z = nullptr;
    int64_t chunk = 0;
};
// Column levels with such a tree (n0 = 3^b0 2^a0) over z rows of P1 x n1 (n1 any length <= 64);
// z needs 2*n0/3 readable rows in front of its first row.
struct Col3Args {
    const float2 *z = nullptr;
    int64_t P1 = 0, rows_out = 0;
    int n1 = 1;
    int b0 = 0, a0 = 0;             // n0 = 3^b0 2^a0
    float2 *out = nullptr;
    float scale = 1.f;
    int64_t chunk = 0;
};
cudaError_t launch_row_tree3(const Row3Args &a, cudaStream_t s);
cudaError_t launch_col_tree3(const Col3Args &a, cudaStream_t s);

cudaError_t launch_adj_col(const AdjColArgs &a, cudaStream_t s);
cudaError_t launch_adj_row(const AdjRowArgs &a, cudaStream_t s);

}  // namespace swdft
