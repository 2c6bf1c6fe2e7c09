/*
 * swdft2d.h -- C ABI of the GB300 (sm_103a) 2D Tree Sliding Window DFT library.
 *
 * The operation (Richardson & Eddy, "The 2D Tree Sliding Window Discrete Fourier
 * Transform", arXiv 1707.08213):
 *
 *   Section 4.1, Eq. (2): for an N0 x N1 array x and n0 x n1 windows (n_i = 2^m_i <= 64,
 *   or 3^b_i 2^a_i <= 64 with b_i >= 1 by ternary and mixed-radix trees; n_i <= N_i), every
 *   window position gets its 2D DFT
 *
 *     a[q0,q1,k0,k1] = c * sum_{j0<n0} sum_{j1<n1} x[q0+j0, q1+j1] w_{n0}^{-j0 k0} w_{n1}^{-j1 k1}
 *
 *   with w_n = exp(2 pi i / n), k_i < n_i, q_i < P_i = N_i - n_i + 1.  The paper names a
 *   window by its last row/column p_i = q_i + n_i - 1 (p_i = n_i-1 .. N_i-1); the
 *   position convention below only chooses which of the two indices the caller uses.
 *   The default scale c is Eq. (2)'s 1/sqrt(n0 n1).
 *
 *   Section 4.2, Eqs. (rowfswft2d), (colfswft2d): the GPU evaluates it with the paper's tree
 *   of radix-2 butterflies shared between overlapping windows, O(N0 N1 n0 n1) work:
 *   m1 levels along dimension 1 (shift s = 2^(m1-t)), then m0 levels along dimension 0
 *   (shift s = 2^(m0+m1-v)), each node T_A = T_B + Omega_C * T_D.  Level m0+m1 is the
 *   window's DFT in natural (k0, k1) order.
 *
 * Memory layout (all row-major, no padding between windows):
 *   input  : N0 rows of N1 elements, row stride ld elements; float32 (SWDFT_R32) or
 *            interleaved complex64 (SWDFT_C64).
 *   output : complex64 interleaved (re, im), [q0 - row_begin][q1][k0][k1]; the window's
 *            n0*n1 coefficients are contiguous, windows of one output row are contiguous.
 *            Bytes = 8 * rows * P1 * n0 * n1.
 *
 * Ownership: the caller owns every input, output and workspace buffer and passes plain
 * pointers; the plan owns only host-side state (twiddle tables, chosen kernels, tuning,
 * a captured CUDA graph and, with SWDFT_FLAG_HOST_IO, device staging buffers).
 * swdft2d_destroy frees only what the plan owns.
 *
 * Errors: every call returns a swdft_status; nothing aborts, exits or throws across the
 * ABI.  Argument checks happen before any CUDA call.  A CUDA launch or copy failure
 * returns SWDFT_ERR_CUDA; asynchronous faults surface at the next synchronising call.
 * The only device-side waits are the tensor-core and TMA-staged kernels' mbarrier waits, the
 * pipelined batch kernels' waits on their row tiles' counters (and the one of
 * swdft2d_selftest_wait_timeout); each gives up after a bounded number of polls or clock
 * cycles and records it (see swdft2d_check_device).
 *
 * Threads and streams: a plan is immutable after swdft2d_plan except for its tuning
 * state, graph and staging buffers; do not execute one plan on two streams at once.
 */
#ifndef SWDFT2D_H
#define SWDFT2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swdft2d_plan_s *swdft2d_plan_t; /* opaque, library-owned */

typedef enum {
    SWDFT_OK = 0,
    SWDFT_ERR_INVALID_ARG = -1,       /* null pointer, bad enum, negative size, bad band */
    SWDFT_ERR_NOT_POW2 = -2,          /* n0 or n1 is neither a power of two (Sec. 4.2's radix-2
                                       * tree) nor 3^b 2^a with b >= 1 (ternary and mixed-radix
                                       * trees) */
    SWDFT_ERR_WINDOW_TOO_LARGE = -3,  /* n_i > N_i: no window position exists */
    SWDFT_ERR_UNSUPPORTED = -4,       /* valid request the library does not implement */
    SWDFT_ERR_OOM = -5,               /* host or device allocation of plan-owned memory failed */
    SWDFT_ERR_CUDA = -6,              /* a CUDA runtime call failed (launch, copy, graph) */
    SWDFT_ERR_DEVICE_TIMEOUT = -7,    /* a bounded device wait ran out (swdft2d_check_device) */
    SWDFT_ERR_WORKSPACE = -8          /* workspace pointer null or misaligned while size > 0 */
} swdft_status;

typedef enum { SWDFT_R32 = 0, SWDFT_C64 = 1 } swdft_dtype;

typedef enum {
    SWDFT_NORM_UNITARY = 0, /* c = 1/sqrt(n0 n1), Eq. (2) (default) */
    SWDFT_NORM_NONE = 1,    /* c = 1, the bare tree sums of Eqs. (rowfswft2d)/(colfswft2d) */
    SWDFT_NORM_INV_N = 2    /* c = 1/(n0 n1), the 2D analogue of the 1D Eq. (1) */
} swdft_norm;

typedef enum {
    SWDFT_POS_START = 0, /* band rows given as q0 = first row of the window */
    SWDFT_POS_END = 1    /* band rows given as p0 = last row of the window (the paper's p) */
} swdft_pos;

typedef enum {
    SWDFT_ALGO_AUTO = 0,          /* tree unless a tuned choice says otherwise */
    SWDFT_ALGO_TREE_F32 = 1,      /* FP32 tree (Section 4.2) on CUDA cores */
    SWDFT_ALGO_TC_BF16X3 = 2,     /* row GEMM + column GEMM on tcgen05, split bf16 hi/lo, 3 terms */
    SWDFT_ALGO_TC_BF16 = 3,       /* same, plain bf16 operands (error reported, not bounded) */
    SWDFT_ALGO_TC_F16_SCALED = 4, /* same, fp16 operands with a per-image scale */
    SWDFT_ALGO_TC_F16 = 5         /* same, plain fp16 operands */
} swdft_algo;

enum {
    SWDFT_FLAG_GRAPH = 1u,    /* capture each execute's launch sequence in a CUDA graph, replay after */
    SWDFT_FLAG_HOST_IO = 2u,  /* plan owns device staging so swdft2d_execute_host can run */
    SWDFT_FLAG_PERSISTENT = 4u, /* batch: one persistent kernel per window shape (n0, n1) over all
                                 * its arrays' tiles -- a pipelined row+column kernel, or a
                                 * fused one for n0 n1 <= 64 -- run concurrently; radix-2 tree only */
    SWDFT_FLAG_AUTOTUNE = 8u    /* the first swdft2d_execute runs swdft2d_autotune on its own
                                 * buffers first (blocking; skipped if its stream is capturing) */
};

/* One array of a batch.  row_begin/row_end select a band of output window rows in the
 * plan's position convention ([row_begin, row_end); row_end = 0 means through the last
 * window row).  The band still reads rows from row 0 of the input pointer. */
typedef struct {
    int64_t N0, N1;  /* array rows and columns, >= 1 */
    int64_t ld;      /* input row stride in elements, >= N1; 0 means N1 */
    int32_t n0, n1;  /* window rows and columns: powers of two (<= 64), or 3^b 2^a <= 64
                      * with b >= 1 (3, 6, 9, 12, 18, 24, 27, 36, 48, 54: ternary and
                      * mixed-radix trees), 1 <= n_i <= N_i; such an n1 needs an n0 of that
                      * kind too (or 1) */
    int32_t dtype;   /* swdft_dtype of the input */
    int32_t reserved;
    int64_t row_begin, row_end;
} swdft2d_shape;

/* Create a plan for `batch` arrays (Section 4.1's problem for each).  Host work only:
 * validates every shape (SWDFT_ERR_NOT_POW2 / WINDOW_TOO_LARGE / INVALID_ARG), builds the
 * twiddle vectors Omega^0, Omega^1 of Section 4.2 in FP64 and rounds them to FP32, and
 * picks kernels.  SWDFT_ERR_UNSUPPORTED for an algorithm or window size the library lacks
 * (tree: n_i <= 64; tensor-core forms: powers of two with 16 <= n0 <= 64 and 8 <= n1 <= 64;
 * ternary and mixed-radix windows: tree only).  With SWDFT_FLAG_PERSISTENT,
 * tensor-core and ternary or mixed-radix arrays run on their own launches beside the
 * persistent kernels (swdft2d_get_form).  *plan is NULL on any error. */
swdft_status swdft2d_plan(swdft2d_plan_t *plan, int32_t batch, const swdft2d_shape *shapes,
                          int32_t norm, int32_t pos, int32_t algo, uint32_t flags);

/* out[4] = {band rows, P1, n0, n1} of array i (Eq. (2)'s P0 x P1 x n0 x n1 output). */
swdft_status swdft2d_output_shape(swdft2d_plan_t plan, int32_t i, int64_t out[4]);

/* Device workspace bytes execute/execute_adjoint need (0 allowed; then pass NULL).
 * The workspace must be 256-byte aligned; its contents need no initialisation. */
swdft_status swdft2d_workspace_size(swdft2d_plan_t plan, size_t *bytes);

/* The algorithm actually used (after AUTO and tuning). */
swdft_status swdft2d_get_algo(swdft2d_plan_t plan, int32_t *algo);

/* How array i runs, after AUTO and tuning: *algo its algorithm (swdft_algo), *form
 * SWDFT_FORM_PIPELINED / SWDFT_FORM_FUSED_GROUP (a persistent plan's kernels shared by the
 * arrays of one window shape) or SWDFT_FORM_PER_ARRAY (its own launches; every array of a
 * plan without SWDFT_FLAG_PERSISTENT).  Either pointer may be NULL.  SWDFT_ERR_INVALID_ARG
 * for a bad plan or index. */
enum { SWDFT_FORM_PIPELINED = 0, SWDFT_FORM_FUSED_GROUP = 1, SWDFT_FORM_PER_ARRAY = 2 };
swdft_status swdft2d_get_form(swdft2d_plan_t plan, int32_t i, int32_t *algo, int32_t *form);

/* Forward transform, Eq. (2), of every array of the plan, enqueued on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  d_in[i] / d_out[i]: device pointers of
 * array i, layouts above; input 4-byte (R32) or 8-byte (C64) aligned, output 16-byte
 * aligned.  d_workspace: swdft2d_workspace_size bytes.  Returns after enqueueing. */
swdft_status swdft2d_execute(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out,
                             void *d_workspace, void *stream);

/* Adjoint A^H of the forward map:
 *   g[r,c] = sum over windows q containing (r,c) of c * sum_k G[q,k] w_{n0}^{+(r-q0)k0} w_{n1}^{+(c-q1)k1}
 * i.e. the overlap-add of every window's inverse DFT of the upstream gradient G: for
 * power-of-two windows the transposed tree (conjugated twiddles), for ternary and
 * mixed-radix windows dense inverse DFTs of length n per window and axis, overlap-added
 * (a power-of-two row window still takes the transposed tree).
 * d_grad_out[i]: complex64 G with the forward output layout (band rows only);
 * d_grad_in[i]: N0 x N1 (row stride N1) float32 = Re(A^H G) for R32 inputs, complex64
 * for C64.  Every element of d_grad_in is written (rows outside the band's reach get 0). */
swdft_status swdft2d_execute_adjoint(swdft2d_plan_t plan, const void *const *d_grad_out,
                                     void *const *d_grad_in, void *d_workspace, void *stream);

/* Forward transform with HOST buffers (plan made with SWDFT_FLAG_HOST_IO): copies each
 * input host->device, runs the transform in output-row bands and copies every band
 * device->host while the next band computes, then synchronises `stream`.  Host buffers
 * should be page-locked (cudaHostAlloc / torch pin_memory) for the copies to overlap. */
swdft_status swdft2d_execute_host(swdft2d_plan_t plan, const void *const *h_in,
                                  void *const *h_out, void *stream);

/* Time every candidate kernel configuration of this plan on the given buffers (CUDA
 * events on `stream`) and keep the fastest; the choice is reused by later executes and
 * recorded in the cache file named by the SWDFT_TUNE_CACHE environment variable, if set
 * (see the tuning cache below).
 * Arrays of the same shape, band and algorithm setting are timed once (the first of them)
 * and share its choice. */
swdft_status swdft2d_autotune(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out,
                              void *d_workspace, void *stream);

/* Tuning cache.  With SWDFT_TUNE_CACHE set, swdft2d_autotune first applies the records that
 * file already holds for this GPU (below) and times only the arrays without one; each array
 * it times appends one line, a JSON object with the GPU name, the array (N0, N1, ld, n0, n1,
 * dtype, q_begin, q_end, whether the plan's algorithm is SWDFT_ALGO_AUTO), the choice
 * (algorithm, fused, row_B, row_chunk, col_B, col_chunk, col_groups) and its time in ms.
 *
 * swdft2d_load_tuning applies such records to a plan without timing anything: each array
 * takes the last record of `path` made on the GPU named `gpu_name` (NULL: the current
 * device's name) for the same array whose choice the plan can run.  *applied (may be NULL)
 * receives the number of arrays set.  A missing file or lines in another layout apply
 * nothing.  Host only when gpu_name is given; SWDFT_ERR_CUDA if the device name is needed
 * and cannot be read. */
swdft_status swdft2d_load_tuning(swdft2d_plan_t plan, const char *path, const char *gpu_name,
                                 int32_t *applied);

/* One pass of the forward tree only, for profiling: stage 0 runs the row levels
 * (Eq. rowfswft2d) of every array into the workspace, stage 1 the column levels
 * (Eq. colfswft2d) from the workspace into d_out.  stage 0 then 1 equals swdft2d_execute
 * (without graph capture).  Other stage values: SWDFT_ERR_INVALID_ARG. */
swdft_status swdft2d_execute_stage(swdft2d_plan_t plan, int32_t stage, const void *const *d_in,
                                   void *const *d_out, void *d_workspace, void *stream);

/* Override the tree kernels' launch configuration of array i (what swdft2d_autotune
 * chooses): row_B / col_B = log2 of the threads sharing one tree's butterflies along
 * dimension 1 / 0 (clamped to [0, min(m, 3)]), row_chunk = window columns per row-pass
 * thread, col_chunk = window rows per column-pass thread (0 = all), col_groups = 32-channel
 * groups per column-pass block, fused = 1: evaluate the row levels inside the column
 * kernel (one launch, z never written to HBM; windows with n1 <= 32, or n1 = 64 and
 * n0 <= 32), 0: two passes, -1: the library's default.  Results do not depend on these
 * values; speed does. */
swdft_status swdft2d_set_tree_config(swdft2d_plan_t plan, int32_t i, int32_t row_B,
                                     int64_t row_chunk, int32_t col_B, int64_t col_chunk,
                                     int32_t col_groups, int32_t fused);

/* Number of kernel launches one execute enqueues (graph replays count their kernels). */
swdft_status swdft2d_launch_count(swdft2d_plan_t plan, int32_t adjoint, int32_t *launches);

/* Forward transform without any allocation, for callers that may not call cudaMalloc
 * (plug-ins handed only their input and output buffers, code running after a framework
 * has claimed the device memory for its own pool, real-time paths where an allocation's
 * latency or failure is not acceptable).  The paper has no counterpart; this is a service
 * of this library.  It needs no plan and no workspace: the z rows between the row-level
 * and column-level passes live in a fixed 32 MiB array of device memory inside the library
 * (held on every GPU that loads it, until exit), and the output is produced in bands of
 * window rows whose z fits there.  Arguments as in swdft2d_shape / swdft2d_execute
 * (ld = 0 means N1); output layout as for swdft2d_execute with all P0 window rows.
 * Radix-2 trees only: windows of 2^m <= 64 per side.  Errors: SWDFT_ERR_UNSUPPORTED for
 * sides of 3^b 2^a samples with b >= 1 (ternary and mixed-radix trees, which plans accept)
 * and for sides above 64; SWDFT_ERR_NOT_POW2 for sides of no such form;
 * otherwise as swdft2d_plan for the shape; SWDFT_ERR_WORKSPACE when even a one-row band
 * needs more than 32 MiB, i.e. (3*n0/2) * (N1-n1+1) * n1 * 8 bytes > 32 MiB.
 * The first call on a device looks up the array's address there and the device's SM count
 * (do it before any stream capture); both are kept until exit, so the entry point must not
 * be used on a device after cudaDeviceReset.  All calls share the array and it keeps the
 * last call's contents: calls that overlap on the GPU race and must be serialised by the
 * caller. */
swdft_status swdft2d_execute_static_scratch(const void *d_in, int64_t N0, int64_t N1, int64_t ld,
                                            int32_t n0, int32_t n1, int32_t dtype, int32_t norm,
                                            void *d_out, void *stream);

/* Device-side health of the current device: SWDFT_ERR_DEVICE_TIMEOUT if, since the last
 * call, a tensor-core kernel, a TMA-staged column kernel or a pipelined batch kernel gave up
 * on one of its bounded waits (its outputs are then incomplete) or
 * swdft2d_selftest_wait_timeout ran; SWDFT_OK otherwise.  Reads and resets
 * the library's device status words (synchronous copies).  SWDFT_ERR_CUDA if a read fails. */
swdft_status swdft2d_check_device(void);

/* Self-test of that time-out path: enqueues on `stream` one block whose thread waits on a
 * shared-memory mbarrier that nothing arrives on, for at most `polls` polls (1..4096; each
 * suspends the thread for at most about 1 ms), then records the time-out in a device
 * status word of its own, read and reset with the tensor-core kernels' word by
 * swdft2d_check_device, which then returns SWDFT_ERR_DEVICE_TIMEOUT.  Nothing faults and
 * the context stays usable.  SWDFT_ERR_INVALID_ARG for polls out of range (checked before
 * any CUDA call). */
swdft_status swdft2d_selftest_wait_timeout(int32_t polls, void *stream);

/* Test hook for the pipelined persistent batch kernels' bounded waits (a column tile waits,
 * spinning on a device counter, until the row tiles of the z rows it reads have finished).
 * budget_cycles: clock64 cycles one column tile may wait before it records a time-out and
 * every block of the launch stops (0 restores the default, about a second); poison: extra
 * row tiles, which never run, that the column tiles of the batch's array 0 wait for (0 in
 * normal use).  A time-out leaves that launch's outputs incomplete and makes the next
 * swdft2d_check_device return SWDFT_ERR_DEVICE_TIMEOUT; nothing faults and the context stays
 * usable.  Process-wide; read when a persistent launch is enqueued or captured into a graph.
 * SWDFT_ERR_INVALID_ARG for negative values. */
swdft_status swdft2d_debug_batch_wait(int64_t budget_cycles, int32_t poison);

/* Fault injection for tests: the library's next `after` allocations succeed and every later
 * one fails with SWDFT_ERR_OOM, until a call with after < 0 turns injection off (the
 * default).  Counted allocations: plan and stream objects (host), a persistent plan's
 * descriptor tables (pinned host and device) and tile table (device), and the device buffers of
 * swdft2d_execute_host.  Process-wide (one atomic counter).  A call that fails this way
 * keeps what it did allocate, so repeating it once injection is off completes it.  Always
 * returns SWDFT_OK. */
swdft_status swdft2d_inject_alloc_failure(int64_t after);

/* Free the plan and everything it owns.  NULL is accepted. */
swdft_status swdft2d_destroy(swdft2d_plan_t plan);

/* Static string for a status code. */
const char *swdft2d_status_string(int32_t status);

/* Library version, major*10000 + minor*100 + patch. */
int32_t swdft2d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWDFT2D_H */
