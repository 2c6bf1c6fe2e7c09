// C-ABI of the k-dimensional transform (include/swdftkd.h; arXiv 1707.08213 Section 4.4,
// Eq. kdfswft).  Host code only: validation, the pass sequence and its workspace layout.
//
// Pass sequence for k >= 3 (dimension d's level group, last dimension first):
//   row pass    : levels of dimension k-1 along every input row (Eq. rowfswft2d's kernel),
//                 Z_{k-1}[r_0..r_{k-2}][q_{k-1}][k_{k-1}];
//   column pass : for d = k-2 .. 0, levels of dimension d (Eq. colfswft2d's kernel) over
//                 the rows r_d of Z_{d+1}, one stack of rows per position of dimensions < d:
//                 Z_d[r_0..r_{d-1}][q_d][q_{d+1}..][k_d][k_{d+1}..].
// Z_0 is the output, scaled.  A column pass sees each row of Z_{d+1} as channels
// (q_{d+1..}, k_{d+1..}) with the coefficient block k_{d+1..} contiguous, exactly the 2D
// column pass's (q1, k1) with n1 replaced by prod_{e>d} n_e, and it writes k_d between the
// position and the block, which is the output order the header specifies.
// k <= 2 runs the 2D plan (k = 1 as a 1 x N_0 array with a 1 x n_0 window).
#include "swdftkd.h"

#include <algorithm>
#include <cmath>
#include <new>

#include "swdft_internal.h"

using namespace swdft;

namespace {

constexpr size_t kKdAlign = 256;
size_t kd_align(size_t v) { return (v + kKdAlign - 1) / kKdAlign * kKdAlign; }

int kd_log2(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while ((int64_t(1) << m) < n) ++m;
    return (int64_t(1) << m) == n ? m : -1;
}

// One column pass (dimension d) of the sequence.
struct KdColPass {
    int d = 0;
    ColTreeArgs args;      // z/out filled in at execute from the workspace offsets
    int src = 0, dst = 0;  // buffer index (0, 1) read / written; dst = -1: the output
    size_t src_pad = 0;    // elements of padding in front of the source rows
    size_t dst_pad = 0;
};

}  // namespace

struct swdftkd_plan_s {
    int k = 0, dtype = SWDFT_R32, norm = SWDFT_NORM_UNITARY;
    int64_t N[SWDFT_KD_MAX_DIMS] = {}, P[SWDFT_KD_MAX_DIMS] = {};
    int n[SWDFT_KD_MAX_DIMS] = {}, m[SWDFT_KD_MAX_DIMS] = {};
    swdft2d_plan_t inner = nullptr;  // k <= 2
    float2 om64[kMaxN];
    RowTreeArgs row;                 // k >= 3: the last dimension's levels
    size_t row_pad = 0;
    KdColPass cols[SWDFT_KD_MAX_DIMS];
    int ncols = 0;
    size_t buf_off[2] = {0, 0};      // byte offsets of the two intermediate buffers
    size_t ws_bytes = 0;
};

namespace {

float kd_scale(int norm, double nn) {
    switch (norm) {
        case SWDFT_NORM_NONE: return 1.0f;
        case SWDFT_NORM_INV_N: return (float)(1.0 / nn);
        default: return (float)(1.0 / std::sqrt(nn));
    }
}

// Chunks of window rows per column pass: enough blocks to fill the GPU several times
// over, never chunks shorter than 2n (the n-1 warm-up steps stay under a third).
int64_t kd_col_chunk(int64_t rows_out, int n, int64_t blocks_per_chunk) {
    constexpr int64_t kTargetBlocks = 152 * 32;
    int64_t nchunks = (kTargetBlocks + blocks_per_chunk - 1) / std::max<int64_t>(1, blocks_per_chunk);
    nchunks = std::min<int64_t>(8, std::max<int64_t>(1, nchunks));
    const int64_t chunk = (rows_out + nchunks - 1) / nchunks;
    return std::min(rows_out, std::max<int64_t>(chunk, 2 * n));
}

swdft_status kd_build_passes(swdftkd_plan_t p) {
    const int K = p->k;
    // row pass: every input row of the last dimension
    int64_t rows = 1;
    for (int e = 0; e < K - 1; ++e) rows *= p->N[e];
    const int ml = p->m[K - 1];
    const int64_t Pl = p->P[K - 1];
    if (rows > INT32_MAX || Pl > INT32_MAX) return SWDFT_ERR_UNSUPPORTED;
    RowTreeArgs &r = p->row;
    r.ld = p->N[K - 1];
    r.cplx = p->dtype == SWDFT_C64;
    r.r_base = 0;
    r.rows = rows;
    r.P1 = Pl;
    r.m1 = ml;
    r.om64 = p->om64;
    r.B = ml >= 6 ? 2 : std::min(ml, 3);
    {
        const int64_t nchunk = std::max<int64_t>(1, (64LL << 10) / std::max<int64_t>(1, rows << r.B));
        const int64_t chunk = (Pl + nchunk - 1) / nchunk;
        r.chunk = std::min<int64_t>(Pl, std::max<int64_t>(chunk, std::max(1, (1 << ml) / 2)));
    }
    // column passes d = K-2 .. 0.  The row pass writes buffer 0; each pass writes the other
    // buffer than it reads, the last one writes the output.  Source rows of pass d hold
    // C = Q << inner channels: Q = prod_{e>d} P_e positions times the 2^inner coefficients
    // of the dimensions after d; a slice (one position of the dimensions before d) is N_d
    // such rows in, P_d rows of C << m_d channels out.
    double nn = 1;
    for (int e = 0; e < K; ++e) nn *= p->n[e];
    size_t need[2] = {0, 0};
    int64_t C = Pl << ml;
    int64_t Q = Pl;
    int inner = ml;
    int src = 0;
    p->row_pad = (size_t)(p->n[K - 2] / 2) * (size_t)C;  // look-back rows of the first column pass
    need[0] = p->row_pad + (size_t)rows * (size_t)C;
    size_t src_pad = p->row_pad;
    p->ncols = 0;
    for (int d = K - 2; d >= 0; --d) {
        if (p->P[d] > INT32_MAX || C > (INT64_MAX >> 8) / std::max<int64_t>(1, p->P[d]))
            return SWDFT_ERR_UNSUPPORTED;
        KdColPass &cp = p->cols[p->ncols++];
        cp.d = d;
        int64_t slices = 1;
        for (int e = 0; e < d; ++e) slices *= p->N[e];
        const int64_t out_row = C << p->m[d];  // channels of one output row
        ColTreeArgs &a = cp.args;
        a.P1 = Q;
        a.rows_out = p->P[d];
        a.m0 = p->m[d];
        a.m1 = inner;
        a.scale = d == 0 ? kd_scale(p->norm, nn) : 1.0f;
        a.om64 = p->om64;
        a.B = a.m0 >= 6 ? 3 : std::min(a.m0, 2);
        a.groups = 1;
        a.slices = slices;
        a.z_slice = p->N[d] * C;
        a.out_slice = p->P[d] * out_row;
        a.chunk = kd_col_chunk(a.rows_out, p->n[d], ((C + 31) / 32) * slices);
        cp.src = src;
        cp.src_pad = src_pad;
        if (d > 0) {
            cp.dst = 1 - src;
            cp.dst_pad = (size_t)(p->n[d - 1] / 2) * (size_t)a.out_slice;  // next pass's look-back
            need[cp.dst] = std::max(need[cp.dst], cp.dst_pad + (size_t)slices * (size_t)a.out_slice);
        } else {
            cp.dst = -1;
            cp.dst_pad = 0;
        }
        Q *= p->P[d];
        inner += p->m[d];
        C = a.out_slice;
        if (d > 0 && inner > kMaxInnerLog2) return SWDFT_ERR_UNSUPPORTED;
        src = cp.dst;
        src_pad = cp.dst_pad;
    }
    p->buf_off[0] = 0;
    p->buf_off[1] = kd_align(need[0] * sizeof(float2));
    p->ws_bytes = p->buf_off[1] + kd_align(need[1] * sizeof(float2));
    return SWDFT_OK;
}

}  // namespace

extern "C" {

swdft_status swdftkd_plan(swdftkd_plan_t *out, const swdftkd_shape *shape, int32_t norm, uint32_t flags) {
    if (!out) return SWDFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!shape || shape->k < 1 || shape->k > SWDFT_KD_MAX_DIMS) return SWDFT_ERR_INVALID_ARG;
    if (shape->dtype != SWDFT_R32 && shape->dtype != SWDFT_C64) return SWDFT_ERR_INVALID_ARG;
    if (norm < SWDFT_NORM_UNITARY || norm > SWDFT_NORM_INV_N) return SWDFT_ERR_INVALID_ARG;
    const int K = shape->k;
    for (int d = 0; d < K; ++d)
        if (shape->N[d] < 1 || shape->n[d] < 1) return SWDFT_ERR_INVALID_ARG;
    for (int d = 0; d < K; ++d)
        if (kd_log2(shape->n[d]) < 0) return SWDFT_ERR_NOT_POW2;
    for (int d = 0; d < K; ++d)
        if (shape->n[d] > shape->N[d]) return SWDFT_ERR_WINDOW_TOO_LARGE;
    for (int d = 0; d < K; ++d)
        if (shape->n[d] > kMaxN) return SWDFT_ERR_UNSUPPORTED;
    if (flags != 0) return SWDFT_ERR_UNSUPPORTED;

    swdftkd_plan_t p = alloc_fails() ? nullptr : new (std::nothrow) swdftkd_plan_s;
    if (!p) return SWDFT_ERR_OOM;
    p->k = K;
    p->dtype = shape->dtype;
    p->norm = norm;
    for (int d = 0; d < K; ++d) {
        p->N[d] = shape->N[d];
        p->n[d] = shape->n[d];
        p->m[d] = kd_log2(shape->n[d]);
        p->P[d] = shape->N[d] - shape->n[d] + 1;
    }
    make_omega(kMaxN, p->om64);
    swdft_status st = SWDFT_OK;
    if (K <= 2) {
        swdft2d_shape s2{};
        s2.N0 = K == 1 ? 1 : p->N[0];
        s2.N1 = p->N[K - 1];
        s2.ld = 0;
        s2.n0 = K == 1 ? 1 : p->n[0];
        s2.n1 = p->n[K - 1];
        s2.dtype = p->dtype;
        st = swdft2d_plan(&p->inner, 1, &s2, norm, SWDFT_POS_START, SWDFT_ALGO_TREE_F32, 0);
        if (st == SWDFT_OK) st = swdft2d_workspace_size(p->inner, &p->ws_bytes);
    } else {
        st = kd_build_passes(p);
    }
    if (st != SWDFT_OK) {
        swdftkd_destroy(p);
        return st;
    }
    *out = p;
    return SWDFT_OK;
}

swdft_status swdftkd_output_shape(swdftkd_plan_t p, int64_t out[2 * SWDFT_KD_MAX_DIMS]) {
    if (!p || !out) return SWDFT_ERR_INVALID_ARG;
    for (int i = 0; i < 2 * SWDFT_KD_MAX_DIMS; ++i) out[i] = 0;
    for (int d = 0; d < p->k; ++d) {
        out[d] = p->P[d];
        out[p->k + d] = p->n[d];
    }
    return SWDFT_OK;
}

swdft_status swdftkd_workspace_size(swdftkd_plan_t p, size_t *bytes) {
    if (!p || !bytes) return SWDFT_ERR_INVALID_ARG;
    *bytes = p->ws_bytes;
    return SWDFT_OK;
}

swdft_status swdftkd_launch_count(swdftkd_plan_t p, int32_t *launches) {
    if (!p || !launches) return SWDFT_ERR_INVALID_ARG;
    if (p->inner) return swdft2d_launch_count(p->inner, 0, launches);
    int32_t total = 1;
    for (int i = 0; i < p->ncols; ++i) total += (int32_t)((p->cols[i].args.slices + 65534) / 65535);
    *launches = total;
    return SWDFT_OK;
}

swdft_status swdftkd_execute(swdftkd_plan_t p, const void *d_in, void *d_out, void *d_ws, void *stream) {
    if (!p || !d_in || !d_out) return SWDFT_ERR_INVALID_ARG;
    if (p->ws_bytes > 0 && (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) % kKdAlign) != 0))
        return SWDFT_ERR_WORKSPACE;
    if (p->inner) {
        const void *in[1] = {d_in};
        void *o[1] = {d_out};
        return swdft2d_execute(p->inner, in, o, d_ws, stream);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float2 *buf[2] = {reinterpret_cast<float2 *>(static_cast<char *>(d_ws) + p->buf_off[0]),
                      reinterpret_cast<float2 *>(static_cast<char *>(d_ws) + p->buf_off[1])};
    RowTreeArgs r = p->row;
    r.x = d_in;
    r.z = buf[0] + p->row_pad;
    if (launch_row_tree(r, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    for (int i = 0; i < p->ncols; ++i) {
        const KdColPass &cp = p->cols[i];
        ColTreeArgs a = cp.args;
        a.z = buf[cp.src] + cp.src_pad;
        a.out = cp.dst < 0 ? static_cast<float2 *>(d_out) : buf[cp.dst] + cp.dst_pad;
        if (launch_col_tree(a, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    }
    return SWDFT_OK;
}

swdft_status swdftkd_destroy(swdftkd_plan_t p) {
    if (!p) return SWDFT_OK;
    if (p->inner) swdft2d_destroy(p->inner);
    delete p;
    return SWDFT_OK;
}

}  // extern "C"
