/*
 * swdftstream.h -- streaming ("real-time order") form of the 2D sliding window DFT
 * (Richardson & Eddy, arXiv 1707.08213): rows of an N1-wide array arrive over time, and
 * each push emits the windows its rows complete.
 *
 * Section 4.3 observes that with the trees innermost the 2D Tree SWDFT suits data that
 * arrive in order: with the tree T kept, a new window costs O(n0 n1).  Here what is kept
 * between pushes is the last n0-1 rows: for n1 <= 32 and pushes of at most 4 n0 rows the
 * input rows themselves (a push
 * copies its rows after them and one launch evaluates the row levels, Eq. rowfswft2d,
 * inside the column tiles of the column levels, Eq. colfswft2d); otherwise level m1 of
 * those rows (their row DFTs, "z": a push runs the row levels on its new rows only, then
 * the column levels over the kept rows and the new ones).  Output of a push: the window
 * rows whose last row arrived in it, [q0][q1][k0][k1] complex64 as in swdft2d.h (q0
 * counted from the first row ever pushed), scaled like swdft2d_execute.  Results are
 * bit-identical to one swdft2d_execute over all rows pushed so far.
 *
 * Cost per push of R rows: the column levels of R + n0 - 1 rows (O(n0 n1) per window once
 * R >= n0; the column levels' warm-up re-evaluates n0-1 rows' worth of nodes per push,
 * which is cheaper on this GPU than reading and writing the column levels' own state,
 * several times larger than the kept rows).
 *
 * Memory: the caller owns a device state buffer of swdft2d_stream_state_size bytes
 * (256-byte aligned, no initialisation) and passes the same buffer to every push of one
 * stream; the stream object owns host-side counters only.  Errors as in swdft2d.h; a push
 * is enqueued on `stream` and returns at once.  One stream object must not be pushed from
 * two CUDA streams at once.
 */
#ifndef SWDFTSTREAM_H
#define SWDFTSTREAM_H

#include "swdft2d.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swdft2d_stream_s *swdft2d_stream_t; /* opaque, library-owned */

/* A stream of rows N1 wide, n0 x n1 windows (powers of two, n1 <= N1, n0, n1 <= 64),
 * input dtype (swdft_dtype), scale (swdft_norm), at most max_rows rows per push (>= 1).
 * SWDFT_ERR_NOT_POW2 / WINDOW_TOO_LARGE / INVALID_ARG / UNSUPPORTED as for swdft2d_plan. */
swdft_status swdft2d_stream_create(swdft2d_stream_t *out, int64_t N1, int32_t n0, int32_t n1,
                                   int32_t dtype, int32_t norm, int64_t max_rows);

/* Bytes of the device state buffer a stream needs. */
swdft_status swdft2d_stream_state_size(swdft2d_stream_t s, size_t *bytes);

/* Push nrows rows (0 <= nrows <= max_rows) of the input, row stride ld elements (0 = N1),
 * device pointer d_rows.  Writes *rows_out window rows (each P1 x n0 x n1 complex64) to
 * d_out: nrows once n0-1 rows have been seen before, fewer while the stream fills.
 * *first_row (optional) = the window row index q0 of the first one. */
swdft_status swdft2d_stream_push(swdft2d_stream_t s, const void *d_rows, int64_t nrows, int64_t ld,
                                 void *d_out, void *d_state, int64_t *rows_out, int64_t *first_row,
                                 void *stream);

/* Rows pushed so far. */
swdft_status swdft2d_stream_rows_seen(swdft2d_stream_t s, int64_t *rows);

/* Forget every row pushed so far (the next push starts a new array). */
swdft_status swdft2d_stream_reset(swdft2d_stream_t s);

/* Free the stream object.  NULL is accepted. */
swdft_status swdft2d_stream_destroy(swdft2d_stream_t s);

#ifdef __cplusplus
}
#endif

#endif /* SWDFTSTREAM_H */
