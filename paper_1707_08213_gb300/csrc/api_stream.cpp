// C-ABI of the streaming form (include/swdftstream.h): rows arrive over time; each push
// evaluates the row levels (Eq. rowfswft2d) and the column levels (Eq. colfswft2d) of the
// windows its rows complete.  Host code only: bookkeeping of the kept rows.
//
// Two forms, chosen at creation (the same bits either way):
//  * n1 <= 32 and pushes of at most 4 n0 rows: the kept rows are INPUT rows; a push copies
//    its rows after them and one fused launch (row levels inside the column tile) emits the
//    completed windows.  Measured on 512-wide rows with 32x32 windows, from a CUDA graph:
//    15.1 / 36.9 us per push of 1 / 32 rows against 15.5 / 38.2 for the z form, and a
//    32x smaller state;
//  * otherwise the kept rows are z rows (level m1, P1*n1 complex64 each); a push runs the
//    row levels of its rows, then the column levels over the kept and new z rows (faster
//    for long pushes: 173 against 186 us per push of 256 rows).
// Device state (caller-owned): `pad` look-back rows, then `cap` kept-row slots.  Slot w
// receives the next pushed row; the n0-1 slots before w are the history.  When a push would
// run past cap, the history moves to slots 0..n0-2 first (one device-to-device copy;
// cap = 2(n0-1) + max_rows keeps source and destination apart).
#include "swdftstream.h"

#include <algorithm>
#include <cmath>
#include <new>

#include "swdft_internal.h"

using namespace swdft;

struct swdft2d_stream_s {
    int64_t N1 = 0, P1 = 0, max_rows = 0;
    int n0 = 1, n1 = 1, m0 = 0, m1 = 0, dtype = SWDFT_R32, norm = SWDFT_NORM_UNITARY;
    float2 om64[kMaxN];
    float scale = 1.f;
    int64_t rows_seen = 0;
    int64_t w = 0;     // next slot to write (after the padding)
    int64_t cap = 0;   // slots after the padding
    int64_t pad = 0;   // look-back rows in front (z form only)
    bool fused = false;  // kept rows are input rows (n1 <= 32)
};

namespace {

int st_log2(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while ((int64_t(1) << m) < n) ++m;
    return (int64_t(1) << m) == n ? m : -1;
}

// bytes of one kept row: an input row (fused form) or a z row
size_t row_bytes(const swdft2d_stream_s *s) {
    return s->fused ? (size_t)s->N1 * (s->dtype == SWDFT_C64 ? sizeof(float2) : sizeof(float))
                    : (size_t)(s->P1 * s->n1) * sizeof(float2);
}

}  // namespace

extern "C" {

swdft_status swdft2d_stream_create(swdft2d_stream_t *out, int64_t N1, int32_t n0, int32_t n1, int32_t dtype,
                                   int32_t norm, int64_t max_rows) {
    if (!out) return SWDFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (N1 < 1 || n0 < 1 || n1 < 1 || max_rows < 1) return SWDFT_ERR_INVALID_ARG;
    if (dtype != SWDFT_R32 && dtype != SWDFT_C64) return SWDFT_ERR_INVALID_ARG;
    if (norm < SWDFT_NORM_UNITARY || norm > SWDFT_NORM_INV_N) return SWDFT_ERR_INVALID_ARG;
    if (st_log2(n0) < 0 || st_log2(n1) < 0) return SWDFT_ERR_NOT_POW2;
    if (n1 > N1) return SWDFT_ERR_WINDOW_TOO_LARGE;
    if (n0 > kMaxN || n1 > kMaxN) return SWDFT_ERR_UNSUPPORTED;
    if (N1 - n1 + 1 > INT32_MAX || max_rows > INT32_MAX / 2) return SWDFT_ERR_UNSUPPORTED;
    swdft2d_stream_t s = alloc_fails() ? nullptr : new (std::nothrow) swdft2d_stream_s;
    if (!s) return SWDFT_ERR_OOM;
    s->N1 = N1;
    s->P1 = N1 - n1 + 1;
    s->max_rows = max_rows;
    s->n0 = n0;
    s->n1 = n1;
    s->m0 = st_log2(n0);
    s->m1 = st_log2(n1);
    s->dtype = dtype;
    s->norm = norm;
    const double nn = (double)n0 * (double)n1;
    s->scale = norm == SWDFT_NORM_NONE ? 1.0f : norm == SWDFT_NORM_INV_N ? (float)(1.0 / nn) : (float)(1.0 / std::sqrt(nn));
    make_omega(kMaxN, s->om64);
    s->fused = s->m1 <= 5 && max_rows <= 4 * (int64_t)n0;
    s->pad = s->fused ? 0 : n0 / 2;  // the fused stage reads look-back rows as zeros
    s->cap = 2 * (int64_t)(n0 - 1) + max_rows;
    *out = s;
    return SWDFT_OK;
}

swdft_status swdft2d_stream_state_size(swdft2d_stream_t s, size_t *bytes) {
    if (!s || !bytes) return SWDFT_ERR_INVALID_ARG;
    *bytes = (size_t)(s->pad + s->cap) * row_bytes(s);
    return SWDFT_OK;
}

swdft_status swdft2d_stream_push(swdft2d_stream_t s, const void *d_rows, int64_t nrows, int64_t ld, void *d_out,
                                 void *d_state, int64_t *rows_out, int64_t *first_row, void *stream) {
    if (!s || !rows_out || nrows < 0 || nrows > s->max_rows) return SWDFT_ERR_INVALID_ARG;
    if (ld == 0) ld = s->N1;
    if (ld < s->N1) return SWDFT_ERR_INVALID_ARG;
    const int64_t hist = std::min<int64_t>(s->rows_seen, s->n0 - 1);
    const int64_t first = std::max<int64_t>(0, s->rows_seen - (s->n0 - 1));
    const int64_t nout = std::max<int64_t>(0, hist + nrows - (s->n0 - 1));
    *rows_out = 0;
    if (first_row) *first_row = first;
    if (nrows == 0) return SWDFT_OK;
    if (!d_rows || (nout > 0 && !d_out)) return SWDFT_ERR_INVALID_ARG;
    if (!d_state || (reinterpret_cast<uintptr_t>(d_state) % 256) != 0) return SWDFT_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t rb = row_bytes(s);
    char *slots = static_cast<char *>(d_state) + (size_t)s->pad * rb;
    if (s->w + nrows > s->cap) {
        // move the history to the front; source rows start at w - hist >= n0 - 1 >= hist
        if (hist > 0 && cudaMemcpyAsync(slots, slots + (size_t)(s->w - hist) * rb, (size_t)hist * rb,
                                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        s->w = hist;
    }
    const int64_t col_chunk = std::min<int64_t>(nout, std::max<int64_t>((nout + 7) / 8, 2 * s->n0));
    if (s->fused) {
        // keep the new input rows after the history, then one launch over the completed windows
        const size_t esz = s->dtype == SWDFT_C64 ? sizeof(float2) : sizeof(float);
        if (cudaMemcpy2DAsync(slots + (size_t)s->w * rb, rb, d_rows, (size_t)ld * esz, rb, (size_t)nrows,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        if (nout > 0) {
            FusedTreeArgs f;
            f.x = slots + (size_t)(s->w - hist) * rb;
            f.ld = s->N1;
            f.cplx = s->dtype == SWDFT_C64;
            f.P1 = s->P1;
            f.rows_out = nout;
            f.m0 = s->m0;
            f.m1 = s->m1;
            f.out = static_cast<float2 *>(d_out);
            f.scale = s->scale;
            f.om64 = s->om64;
            f.chunk = col_chunk;
            f.groups = 1;
            if (launch_fused_tree(f, st) != cudaSuccess) return SWDFT_ERR_CUDA;
        }
    } else {
        const int64_t re = s->P1 * s->n1;
        float2 *z = reinterpret_cast<float2 *>(slots);
        RowTreeArgs r;
        r.x = d_rows;
        r.ld = ld;
        r.cplx = s->dtype == SWDFT_C64;
        r.r_base = 0;
        r.rows = nrows;
        r.P1 = s->P1;
        r.m1 = s->m1;
        r.z = z + s->w * re;
        r.om64 = s->om64;
        r.B = s->m1 >= 6 ? 2 : std::min(s->m1, 3);
        {
            const int64_t nchunk = std::max<int64_t>(1, (64LL << 10) / std::max<int64_t>(1, nrows << r.B));
            const int64_t chunk = (s->P1 + nchunk - 1) / nchunk;
            r.chunk = std::min<int64_t>(s->P1, std::max<int64_t>(chunk, std::max(1, s->n1 / 2)));
        }
        if (launch_row_tree(r, st) != cudaSuccess) return SWDFT_ERR_CUDA;
        if (nout > 0) {
            ColTreeArgs c;
            c.z = z + (s->w - hist) * re;
            c.P1 = s->P1;
            c.rows_out = nout;
            c.m0 = s->m0;
            c.m1 = s->m1;
            c.out = static_cast<float2 *>(d_out);
            c.scale = s->scale;
            c.om64 = s->om64;
            c.B = s->m0 >= 6 ? 3 : std::min(s->m0, 2);
            c.chunk = col_chunk;
            c.groups = 1;
            if (launch_col_tree(c, st) != cudaSuccess) return SWDFT_ERR_CUDA;
        }
    }
    s->w += nrows;
    s->rows_seen += nrows;
    *rows_out = nout;
    return SWDFT_OK;
}

swdft_status swdft2d_stream_rows_seen(swdft2d_stream_t s, int64_t *rows) {
    if (!s || !rows) return SWDFT_ERR_INVALID_ARG;
    *rows = s->rows_seen;
    return SWDFT_OK;
}

swdft_status swdft2d_stream_reset(swdft2d_stream_t s) {
    if (!s) return SWDFT_ERR_INVALID_ARG;
    s->rows_seen = 0;
    s->w = 0;
    return SWDFT_OK;
}

swdft_status swdft2d_stream_destroy(swdft2d_stream_t s) {
    delete s;
    return SWDFT_OK;
}

}  // extern "C"
