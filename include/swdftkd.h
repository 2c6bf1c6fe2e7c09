/*
 * swdftkd.h -- C ABI of the k-dimensional sliding window DFT (k = 1..4), the extension of
 * the 2D Tree SWDFT (Richardson & Eddy, arXiv 1707.08213) given in Section 4.4.
 *
 * The operation: for an N_0 x ... x N_{k-1} array x and n_0 x ... x n_{k-1} windows
 * (n_d = 2^m_d, 1 <= n_d <= N_d), every window position gets its k-dimensional DFT,
 * Eq. (2) with one sum per dimension:
 *
 *   a[q; k] = c * sum_{j_0<n_0} ... sum_{j_{k-1}<n_{k-1}} x[q_0+j_0, ..., q_{k-1}+j_{k-1}]
 *                 * prod_d w_{n_d}^{-j_d k_d},             w_n = exp(2 pi i / n),
 *
 * q_d < P_d = N_d - n_d + 1, k_d < n_d; c = 1/sqrt(prod n_d) by default (swdft_norm).
 * Section 4.4, Eq. (kdfswft): the tree's levels come in groups, one per dimension, the last
 * dimension's m_{k-1} levels first and dimension 0's last; a level of dimension c combines
 * the tree at p with the tree at p - s e_c.  The GPU evaluates the group of the last
 * dimension along every input row, then each earlier dimension's group as one column pass
 * over the previous group's result (for k <= 2 it runs the 2D plan of swdft2d.h).
 *
 * Memory layout (row-major, no padding):
 *   input  : float32 (SWDFT_R32) or interleaved complex64 (SWDFT_C64), [r_0]...[r_{k-1}],
 *            element (r_0..r_{k-1}) at sum_d r_d * prod_{e>d} N_e, 4- / 8-byte aligned.
 *   output : complex64, [q_0]...[q_{k-1}][k_0]...[k_{k-1}], 16-byte aligned;
 *            bytes = 8 * prod P_d * prod n_d.
 *
 * Ownership, errors, streams: as in swdft2d.h.  The caller owns input, output and workspace;
 * the plan owns host state only.  Every call returns a swdft_status and nothing aborts.
 * Arguments are checked before any CUDA call.  A plan must not run on two streams at once.
 */
#ifndef SWDFTKD_H
#define SWDFTKD_H

#include "swdft2d.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SWDFT_KD_MAX_DIMS 4

typedef struct swdftkd_plan_s *swdftkd_plan_t; /* opaque, library-owned */

typedef struct {
    int32_t k;                     /* dimensions, 1..SWDFT_KD_MAX_DIMS */
    int32_t dtype;                 /* swdft_dtype of the input */
    int64_t N[SWDFT_KD_MAX_DIMS];  /* extents, N[k-1] varies fastest; entries >= k ignored */
    int32_t n[SWDFT_KD_MAX_DIMS];  /* window lengths, powers of two, 1 <= n[d] <= N[d], <= 64 */
} swdftkd_shape;

/* Create a plan.  Host work only: validates the shape (SWDFT_ERR_INVALID_ARG for k out of
 * range, an extent < 1 or a bad dtype/norm; SWDFT_ERR_NOT_POW2; SWDFT_ERR_WINDOW_TOO_LARGE;
 * SWDFT_ERR_UNSUPPORTED for n[d] > 64, an output or intermediate beyond 2^31 rows or
 * channels, or flags other than 0), builds Omega of Section 4.2 in FP64 rounded to FP32 and
 * picks the kernels' launch shapes.  *plan is NULL on any error. */
swdft_status swdftkd_plan(swdftkd_plan_t *plan, const swdftkd_shape *shape, int32_t norm,
                          uint32_t flags);

/* out[0..k-1] = P_0..P_{k-1}, out[k..2k-1] = n_0..n_{k-1}; entries from 2k on are 0.
 * out holds 2 * SWDFT_KD_MAX_DIMS entries. */
swdft_status swdftkd_output_shape(swdftkd_plan_t plan, int64_t out[2 * SWDFT_KD_MAX_DIMS]);

/* Device workspace bytes swdftkd_execute needs: the results of the level groups before the
 * last, complex64, 1/n_0 of the output and less (256-byte aligned; no initialisation). */
swdft_status swdftkd_workspace_size(swdftkd_plan_t plan, size_t *bytes);

/* Kernel launches one execute enqueues (k for k >= 3; as the 2D plan for k <= 2). */
swdft_status swdftkd_launch_count(swdftkd_plan_t plan, int32_t *launches);

/* Forward transform of one array, enqueued on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  d_in, d_out, d_workspace: device pointers, layouts above.  Returns
 * after enqueueing; SWDFT_ERR_WORKSPACE if the workspace is NULL or not 256-byte aligned
 * while its size is nonzero; SWDFT_ERR_CUDA if a launch fails. */
swdft_status swdftkd_execute(swdftkd_plan_t plan, const void *d_in, void *d_out,
                             void *d_workspace, void *stream);

/* Free the plan.  NULL is accepted. */
swdft_status swdftkd_destroy(swdftkd_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* SWDFTKD_H */
