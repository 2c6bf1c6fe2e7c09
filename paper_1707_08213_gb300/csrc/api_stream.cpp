// C-ABI of the streaming form (include/swdftstream.h): rows arrive over time; each push
// runs the row levels (Eq. rowfswft2d) of its rows and the column levels (Eq. colfswft2d)
// of the windows they complete.  Host code only: bookkeeping of the kept z rows.
//
// Device state (caller-owned): n0/2 look-back rows, then `cap` z rows of P1*n1 complex64.
// z row w holds the next pushed row's DFTs; the n0-1 rows before w are the kept history.
// When a push would run past cap, the history moves to rows 0..n0-2 first (one
// device-to-device copy; cap = 2(n0-1) + max_rows keeps source and destination apart).
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
    int64_t w = 0;     // next z row to write (after the padding)
    int64_t cap = 0;   // z rows after the padding
    int64_t pad = 0;   // look-back rows in front
};

namespace {

int st_log2(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while ((int64_t(1) << m) < n) ++m;
    return (int64_t(1) << m) == n ? m : -1;
}

int64_t row_elems(const swdft2d_stream_s *s) { return s->P1 * s->n1; }

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
    swdft2d_stream_t s = new (std::nothrow) swdft2d_stream_s;
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
    s->pad = n0 / 2;
    s->cap = 2 * (int64_t)(n0 - 1) + max_rows;
    *out = s;
    return SWDFT_OK;
}

swdft_status swdft2d_stream_state_size(swdft2d_stream_t s, size_t *bytes) {
    if (!s || !bytes) return SWDFT_ERR_INVALID_ARG;
    *bytes = (size_t)(s->pad + s->cap) * (size_t)row_elems(s) * sizeof(float2);
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
    const int64_t re = row_elems(s);
    float2 *z = static_cast<float2 *>(d_state) + s->pad * re;
    if (s->w + nrows > s->cap) {
        // move the history to the front; source rows start at w - hist >= n0 - 1 >= hist
        if (hist > 0 && cudaMemcpyAsync(z, z + (s->w - hist) * re, (size_t)(hist * re) * sizeof(float2),
                                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        s->w = hist;
    }
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
        c.chunk = std::min<int64_t>(nout, std::max<int64_t>((nout + 7) / 8, 2 * s->n0));
        c.groups = 1;
        if (launch_col_tree(c, st) != cudaSuccess) return SWDFT_ERR_CUDA;
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
