// C-ABI of the sliding window DFT library (include/swdft2d.h): plan validation, twiddle
// tables, kernel selection, launch sequencing, CUDA-graph replay, the host-buffer band
// pipeline and the autotuner.  Compute happens only in the kernels of the .cu files.
#include "swdft2d.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "swdft_internal.h"

namespace swdft {
// allocations that may still succeed before injected failures; -1: no injection
static std::atomic<int64_t> g_alloc_budget{-1};

bool alloc_fails() {
    int64_t v = g_alloc_budget.load(std::memory_order_relaxed);
    while (v > 0)
        if (g_alloc_budget.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return false;
    return v == 0;
}
// pipelined batch launches: clock64 cycles a column tile may wait (about a second at the
// GB300's clock), and the test hook's extra row-tile count (swdft2d_debug_batch_wait)
constexpr int64_t kPipeBudget = 2000000000LL;
static std::atomic<int64_t> g_pipe_budget{kPipeBudget};
static std::atomic<int32_t> g_pipe_poison{0};
}  // namespace swdft

using namespace swdft;

namespace {

constexpr size_t kAlign = 256;
// arrays of one plan that run at once on plan-owned streams (per-array launches and the
// adjoint); each has its own workspace slot
constexpr int kConc = 4;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// n = 3^b 2^a with b >= 1 (a ternary or mixed-radix window side): true, and b, a
bool mixed_split(int64_t n, int *b, int *a) {
    if (n < 3) return false;
    int bb = 0, aa = 0;
    while (n % 3 == 0) {
        n /= 3;
        ++bb;
    }
    while (n % 2 == 0) {
        n /= 2;
        ++aa;
    }
    if (n != 1 || bb == 0) return false;
    *b = bb;
    *a = aa;
    return true;
}

int log2_exact(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while ((int64_t(1) << m) < n) ++m;
    return (int64_t(1) << m) == n ? m : -1;
}

struct TreeConfig {
    bool fused = false;  // n1 <= 64: row levels inside the column kernel (no z in HBM)
    int row_B = 2;
    int64_t row_chunk = 0;
    int col_B = 2;
    int64_t col_chunk = 0;
    int col_groups = 2;
};

struct ArrayPlan {
    int64_t N0 = 0, N1 = 0, ld = 0, P0 = 0, P1 = 0;
    int n0 = 1, n1 = 1, m0 = 0, m1 = 0, dtype = SWDFT_R32;
    // radix family of each axis's tree: 2 (n_i = 2^m_i; n_i = 1 counts as radix 2) or 3
    // (n_i = 3^b_i 2^a_i, b_i >= 1: ternary and mixed-radix trees; m_i = b_i)
    int r0 = 2, r1 = 2;
    int b0 = 0, a0 = 0, b1 = 0, a1 = 0;
    int64_t q_begin = 0, q_end = 0;  // band of window rows, q coordinates
    TreeConfig cfg;
    bool tuned = false;
    int algo = SWDFT_ALGO_TREE_F32;  // per array: tree or one of the tensor-core forms
    bool algo_auto = false;          // made with SWDFT_ALGO_AUTO: the autotuner may pick a form
    // persistent batch: how the array runs -- in the pipelined kernel of its window shape,
    // in the fused group of its window shape (no row tiles, no z), or on its own through the
    // per-array launches (tree or tensor-core form) beside the persistent kernels
    int batch_mode = 0;
    int64_t tc_chunk = 48;           // window rows per tensor-core CTA
    // column tiles of the pipelined persistent kernel when cfg is the fused form (whose own
    // chunks are cut for recomputing z): the two-pass rule's chunk
    int64_t pipe_col_chunk = 0;

    int64_t band_rows() const { return q_end - q_begin; }
    size_t in_elem() const { return dtype == SWDFT_C64 ? sizeof(float2) : sizeof(float); }
    size_t out_row_bytes() const { return (size_t)P1 * n0 * n1 * sizeof(float2); }
    bool ternary() const { return r0 == 3 || r1 == 3; }
    // padding rows in front of z for the column pass's level-0 look-back (n0/2 for a binary
    // column tree, 2*n0/3 for a ternary one), then rows_out + n0 - 1 rows
    int64_t z_pad() const { return r0 == 3 ? 2 * n0 / 3 : n0 / 2; }
    size_t z_bytes(int64_t rows_out) const {
        return (size_t)(z_pad() + rows_out + n0 - 1) * (size_t)P1 * n1 * sizeof(float2);
    }
    // tensor-core forms: 16-bit operand planes of z after the z buffer, then a max-abs word
    bool tc_eligible() const { return !ternary() && m0 >= 4 && m0 <= 6 && m1 >= 3 && m1 <= 6; }
    static int tc_terms(int algo) { return algo == SWDFT_ALGO_TC_BF16X3 ? 3 : 1; }
    size_t planes_bytes(int64_t rows_out, int algo) const {
        return (size_t)tc_terms(algo) * 2 * (size_t)(rows_out + n0 - 1) * (size_t)P1 * n1 * 2;
    }
    // adjoint: window rows per adj_col chunk (at most eight chunks, none shorter than 6*n0:
    // chunks read disjoint rows of G, and each costs n0-1 drain steps and n0-1 side rows,
    // which a second launch folds into gz; 6*n0 measured up to 8% faster than 4*n0 for
    // n0 >= 32 and the same below), gz where the forward pass keeps z, then the
    // chunks' side rows.  It depends on the array's shape only, so an array's adjoint has
    // the same bits in every plan.
    int64_t adj_chunk(int64_t rows_out) const {
        return std::min(rows_out, std::max<int64_t>((rows_out + 7) / 8, 6 * n0));
    }
    size_t adj_side_bytes(int64_t rows_out) const {
        if (ternary()) return 0;  // the ternary adjoint's chunks share rows through atomics
        return (size_t)adj_side_elems(rows_out, m0, P1, m1, adj_chunk(rows_out)) * sizeof(float2);
    }
    size_t adj_bytes(int64_t rows_out) const { return align_up(z_bytes(rows_out)) + align_up(adj_side_bytes(rows_out)); }
    size_t ws_bytes_for(int64_t rows_out, int algo) const {
        // tree: z (complex64); tensor-core forms: z as operand planes, then a max-abs word;
        // either way at least what the adjoint needs
        const size_t fwd = algo >= SWDFT_ALGO_TC_BF16X3 ? align_up(planes_bytes(rows_out, algo)) + kAlign
                                                        : align_up(z_bytes(rows_out));
        return std::max(fwd, adj_bytes(rows_out));
    }
    // the workspace a plan reserves: room for the split-bf16 form too when the autotuner may
    // choose it
    size_t ws_bytes_plan(int64_t rows_out) const {
        size_t w = ws_bytes_for(rows_out, algo);
        if (algo_auto && tc_eligible()) w = std::max(w, ws_bytes_for(rows_out, SWDFT_ALGO_TC_BF16X3));
        return w;
    }
};

constexpr int kBatchPipe = 0, kBatchFused = 1, kBatchSolo = 2;

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;
    cudaStream_t stream = nullptr;
};

}  // namespace

struct swdft2d_plan_s {
    std::vector<ArrayPlan> arrays;
    int norm = SWDFT_NORM_UNITARY, pos = SWDFT_POS_START, algo = SWDFT_ALGO_TREE_F32;
    uint32_t flags = 0;
    size_t ws_bytes = 0;
    // Omega of length 64 (FP64-evaluated, FP32-rounded): Omega^i of Section 4.2 for every
    // n_i = 2^m_i <= 64 is its strided view, Omega^i[j] = om64[j * 64 / n_i], bit for bit.
    float2 om64[kMaxN];
    bool configured = false;
    bool autotuned = false;  // SWDFT_FLAG_AUTOTUNE: the first execute has tuned the plan
    int sm_count = 152;
    GraphCache graph;
    // several arrays (not persistent): up to kConc of them run concurrently on plan-owned
    // streams forked from and joined back to the caller's stream, one workspace slot each
    int conc = 1;
    size_t slot_bytes = 0;
    // all arrays of one shape and band (not persistent): the adjoint runs groups of up to
    // kAdjZ arrays per launch, each array in its own workspace slot
    bool uniform = false;
    cudaStream_t side[kConc] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kConc] = {};
    // persistent batch (SWDFT_FLAG_PERSISTENT): per-array z offsets in the workspace, the
    // tile descriptors (pinned staging + device copy, allocated at the first execute)
    std::vector<size_t> z_off;
    // descriptor buffers: BatchImage[n], then the fused groups' entries (each group
    // contiguous); pinned staging, a direct-execute copy, a graph copy
    unsigned char *desc_host = nullptr;
    unsigned char *desc_dev = nullptr;
    unsigned char *desc_graph = nullptr;
    size_t desc_bytes = 0;
    cudaEvent_t desc_uploaded = nullptr;
    // fused groups, index m0 * kBatchFusedM1 + m1, on their own side streams
    static constexpr int kFz = (kMaxLog2 + 1) * kBatchFusedM1;
    int fz_off[kFz] = {}, fz_n[kFz] = {};
    int64_t fz_items[kFz] = {}, fz_slots[kFz] = {};
    cudaStream_t fside[kConc] = {};
    cudaEvent_t fjoin_ev[kConc] = {};
    // pipelined classes (every two-pass array of a persistent plan), index m0 * 7 + m1: the
    // class's tiles are items [pz_off, pz_off + pz_n) of the plan-constant item table on the
    // device (pipe_dev).  The workspace ends with the launch's counters: a ticket per class
    // and the abort word (kPipeHead ints), then a flag per (array, row block, row chunk).
    static constexpr int kPz = (kMaxLog2 + 1) * (kMaxLog2 + 1);
    static constexpr int kPipeHead = 64;
    int pz_off[kPz] = {}, pz_n[kPz] = {};
    int64_t pz_slots[kPz] = {};
    int pipe_flags = 0;          // row tiles of all two-pass arrays
    size_t sync_off = 0;         // counters' offset in the workspace
    size_t sync_bytes = 0;
    unsigned char *pipe_dev = nullptr;
    size_t pipe_dev_bytes = 0;
    bool pipe_uploaded = false;  // cleared when the arrays' chunks change (autotuning)
    std::vector<int> pipe_sync;  // per array: its first row-tile flag
    // host-buffer pipeline (SWDFT_FLAG_HOST_IO), allocated at the first execute_host
    bool io_ready = false;
    int64_t io_band = 0;
    void *io_in = nullptr;
    void *io_ws = nullptr;
    void *io_out[2] = {nullptr, nullptr};
    cudaStream_t io_copy = nullptr;
    cudaEvent_t io_done[2] = {nullptr, nullptr};
    cudaEvent_t io_copied[2] = {nullptr, nullptr};
};

namespace {

float norm_scale(int norm, int n0, int n1) {
    const double nn = (double)n0 * (double)n1;
    switch (norm) {
        case SWDFT_NORM_NONE: return 1.0f;
        case SWDFT_NORM_INV_N: return (float)(1.0 / nn);
        default: return (float)(1.0 / std::sqrt(nn));
    }
}

// Column-pass row chunks (default_col_nchunks / default_col_chunk in swdft_internal.h).
int64_t col_chunk_for(const ArrayPlan &a, int nchunks) { return default_col_chunk(a.band_rows(), a.n0, nchunks); }

int col_nchunks(const ArrayPlan &a, int sm_count, bool fused_small) {
    return default_col_nchunks(a.P1 * a.n1, sm_count, fused_small);
}

// conc: arrays of the plan that run at once (their z buffers share L2).
void default_config(ArrayPlan &a, int sm_count, int conc) {
    TreeConfig c;
    // row levels: thread = (row, residue, chunk of window columns).  About 64K threads in
    // flight (measured best on the 512x512/32x32 and 1024x2048/16x64 workloads: B = 3 with
    // 16-32 column chunks, B = 2 with 128-column chunks), chunks no shorter than n1/2.
    c.row_B = a.r1 == 3 ? 0 : default_row_B(a.m1);  // ternary rows: one thread each
    const int64_t rows = a.band_rows() + a.n0 - 1;
    const int64_t per_row = a.r1 == 3 ? (a.m1 >= 1 ? 3 : 1) : (int64_t(1) << c.row_B);  // threads per row
    c.row_chunk = default_row_chunk(a.P1, rows, per_row, a.n1);
    // column levels: thread = (channel, residue, chunk of output rows); one 32-channel
    // group per block (32 * 2^B threads)
    c.col_B = default_col_B(a.m0);
    c.col_groups = 1;
    // fused form (row levels inside the column tile, fused_supported): it recomputes each z value
    // from the input (log2 n1 butterflies) instead of writing and re-reading z, which wins for
    // small windows (z is 1/n0 of the output) and when the z of the arrays in flight would
    // not stay in L2 (measured on 256..1024-square arrays with the 4x4 .. 64x16 windows:
    // fused faster for n0 n1 <= 64 everywhere and for n0 >= 16 once z exceeds ~100 MB)
    const bool can_fuse = !a.ternary() && fused_supported(a.m0, a.m1) && a.algo == SWDFT_ALGO_TREE_F32;
    const bool small = a.n0 * a.n1 <= 64;
    const double z_live = (double)a.z_bytes(a.band_rows()) * std::max(1, conc);
    c.fused = can_fuse && (small || (a.n0 >= 16 && z_live > 96e6));
    // chunks of window rows (col_nchunks); col_chunk_for keeps every chunk at 2 n0 rows or more.
    // The fused form of larger windows recomputes its n0 - 1 warm-up z rows per chunk by row
    // DFTs, so it takes two chunks, more only where few 32-channel groups need them for four
    // blocks per SM (1024x2048 complex, 16x64 windows: 2.585 ms at eight chunks, 2.53 at two).
    int nchunks = col_nchunks(a, sm_count, c.fused && small);
    if (c.fused && !small) {
        const int64_t groups = (a.P1 * a.n1 + 31) / 32;
        nchunks = (int)std::min<int64_t>(nchunks, std::max<int64_t>(2, (4LL * sm_count + groups - 1) / groups));
    }
    c.col_chunk = col_chunk_for(a, nchunks);
    a.pipe_col_chunk = col_chunk_for(a, col_nchunks(a, sm_count, false));
    a.cfg = c;
}

// Tile geometry of a two-pass array in a pipelined persistent launch; the item table built at
// configure time and the descriptors filled per buffer set both come from here.
struct PipeGeom {
    int rpb = 1, row_chunk = 1, row_chunks = 1, row_blocks = 1;
    int col_chunk = 1, col_chunks = 1, col_blocks = 1;
};
PipeGeom pipe_geom(const ArrayPlan &a) {
    PipeGeom g;
    const int64_t rows_out = a.band_rows();
    const int64_t zrows = rows_out + a.n0 - 1;
    g.rpb = batch_pipe_rows_per_tile(a.m0, a.m1);  // row tiles: independent of the tuning state
    g.row_chunk = (int)std::min<int64_t>(
        a.P1, std::max<int64_t>(1, default_row_chunk(a.P1, zrows, int64_t(1) << batch_pipe_row_B(a.m1), a.n1)));
    g.row_chunks = (int)((a.P1 + g.row_chunk - 1) / g.row_chunk);
    g.row_blocks = (int)((zrows + g.rpb - 1) / g.rpb);
    const int64_t cc = a.cfg.fused && a.pipe_col_chunk > 0 ? a.pipe_col_chunk : a.cfg.col_chunk;
    g.col_chunk = (int)std::min<int64_t>(rows_out, std::max<int64_t>(1, cc));
    g.col_chunks = (int)((rows_out + g.col_chunk - 1) / g.col_chunk);
    const int64_t per_block = 32LL * batch_col_groups(a.m0);
    g.col_blocks = (int)((a.P1 * a.n1 + per_block - 1) / per_block);
    return g;
}

// The pipelined classes' tiles in ticket order.  A class's arrays (largest first) are cut
// into stages: per column chunk, the row tiles of the z rows it is the first chunk to read,
// then its column tiles.  Stages keep their order, but each stage's column tiles are held
// back until at least `slots` tickets (the blocks the kernel keeps resident) have been issued
// since its last row tile -- later stages' row tiles, of this array or the next ones, fill
// the gap -- so that when a block takes a column tile its row tiles have almost surely
// finished and the wait is a formality.  The next stage's row tiles always precede a stage's
// column tiles; beyond that at most kPipeZAhead bytes of z are written ahead of their readers,
// so they are still in L2 when read.
constexpr int64_t kPipeZAhead = 48LL << 20;

void build_pipe(swdft2d_plan_s *plan, std::vector<BatchPipeItem> &items, std::vector<int> &sync_off) {
    const size_t n = plan->arrays.size();
    items.clear();
    sync_off.assign(n, 0);
    int off = 0;
    for (size_t i = 0; i < n; ++i) {
        const PipeGeom g = pipe_geom(plan->arrays[i]);
        sync_off[i] = off;
        off += g.row_blocks * g.row_chunks;
    }
    struct Stage {
        int img, rb0, rb1, ck;
        int64_t zbytes;
    };
    for (int c = 0; c < swdft2d_plan_s::kPz; ++c) {
        plan->pz_off[c] = (int)items.size();
        std::vector<size_t> idx;
        for (size_t i = 0; i < n; ++i) {
            const ArrayPlan &a = plan->arrays[i];
            if (a.batch_mode == kBatchPipe && a.m0 * (kMaxLog2 + 1) + a.m1 == c) idx.push_back(i);
        }
        std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
            const ArrayPlan &a = plan->arrays[x], &b = plan->arrays[y];
            return a.band_rows() * a.out_row_bytes() > b.band_rows() * b.out_row_bytes();
        });
        std::vector<Stage> st;
        for (size_t i : idx) {
            const ArrayPlan &a = plan->arrays[i];
            const PipeGeom g = pipe_geom(a);
            const int zrows = (int)(a.band_rows() + a.n0 - 1);
            int next_rb = 0;
            for (int ck = 0; ck < g.col_chunks; ++ck) {
                int r_lo = 0, r_hi = 0;
                pipe_col_rows(ck, g.col_chunk, (int)a.band_rows(), a.n0, &r_lo, &r_hi);
                const int rb1 = std::max(next_rb, (r_hi - 1) / g.rpb + 1);
                const int64_t rows = std::min(rb1 * g.rpb, zrows) - std::min(next_rb * g.rpb, zrows);
                st.push_back({(int)i, next_rb, rb1, ck, rows * a.P1 * a.n1 * (int64_t)sizeof(float2)});
                next_rb = rb1;
            }
        }
        const size_t slots = (size_t)std::max<int64_t>(1, plan->pz_slots[c]);
        std::vector<size_t> dep_end(st.size(), 0);
        int64_t z_ahead = 0;
        size_t r = 0;
        auto emit_rows = [&](size_t k) {
            const Stage &e = st[k];
            const int row_chunks = pipe_geom(plan->arrays[(size_t)e.img]).row_chunks;
            for (int rb = e.rb0; rb < e.rb1; ++rb)
                for (int rc = 0; rc < row_chunks; ++rc) items.push_back({e.img, rb * row_chunks + rc});
            dep_end[k] = items.size();
            z_ahead += e.zbytes;
        };
        for (size_t k = 0; k < st.size(); ++k) {
            while (r <= k + 1 && r < st.size()) emit_rows(r++);  // the next stage's row tiles always go first
            while (r < st.size() && items.size() - dep_end[k] < slots && z_ahead + st[r].zbytes <= kPipeZAhead)
                emit_rows(r++);
            const int col_blocks = pipe_geom(plan->arrays[(size_t)st[k].img]).col_blocks;
            for (int cb = 0; cb < col_blocks; ++cb) items.push_back({st[k].img, ~(st[k].ck * col_blocks + cb)});
            z_ahead -= st[k].zbytes;
        }
        plan->pz_n[c] = (int)items.size() - plan->pz_off[c];
    }
}

swdft_status configure(swdft2d_plan_t plan) {
    if (plan->configured) return SWDFT_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWDFT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SWDFT_ERR_CUDA;
    plan->sm_count = sms > 0 ? sms : 152;
    for (auto &a : plan->arrays)
        if (!a.tuned) default_config(a, plan->sm_count, plan->conc);
    // every object below is created once: a configure that failed part way (out of memory)
    // keeps what it made, the plan's destroy frees it, and the next call resumes
    if (plan->conc > 1) {
        if (!plan->fork_ev && cudaEventCreateWithFlags(&plan->fork_ev, cudaEventDisableTiming) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        for (int k = 0; k < plan->conc; ++k) {
            if (!plan->side[k] && cudaStreamCreateWithFlags(&plan->side[k], cudaStreamNonBlocking) != cudaSuccess)
                return SWDFT_ERR_CUDA;
            if (!plan->join_ev[k] && cudaEventCreateWithFlags(&plan->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
                return SWDFT_ERR_CUDA;
        }
    }
    if (plan->flags & SWDFT_FLAG_PERSISTENT) {
        const size_t n = plan->arrays.size();
        plan->desc_bytes = sizeof(BatchImage) * n + sizeof(BatchClassEntry) * n;
        if (!plan->desc_host && (alloc_fails() || cudaHostAlloc((void **)&plan->desc_host, plan->desc_bytes,
                                                                cudaHostAllocDefault) != cudaSuccess))
            return SWDFT_ERR_OOM;
        if (!plan->desc_dev && (alloc_fails() || cudaMalloc((void **)&plan->desc_dev, plan->desc_bytes) != cudaSuccess))
            return SWDFT_ERR_OOM;
        if (!plan->desc_graph &&
            (alloc_fails() || cudaMalloc((void **)&plan->desc_graph, plan->desc_bytes) != cudaSuccess))
            return SWDFT_ERR_OOM;
        if (!plan->desc_uploaded && cudaEventCreateWithFlags(&plan->desc_uploaded, cudaEventDisableTiming) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        // grid slots of every kernel an array may run in (the autotuner may move arrays
        // between the pipelined and fused kernels)
        for (const auto &a : plan->arrays) {
            const int c = a.m0 * (kMaxLog2 + 1) + a.m1;
            if (plan->pz_slots[c] == 0) {
                int bps = 0;
                if (batch_pipe_blocks_per_sm(a.m0, a.m1, &bps) != cudaSuccess) return SWDFT_ERR_CUDA;
                plan->pz_slots[c] = (int64_t)plan->sm_count * std::max(1, bps);
            }
            if (a.m1 >= kBatchFusedM1) continue;
            const int f = a.m0 * kBatchFusedM1 + a.m1;
            if (plan->fz_slots[f] > 0) continue;
            int bps = 0;
            if (batch_fused_blocks_per_sm(a.m0, a.m1, &bps) != cudaSuccess) return SWDFT_ERR_CUDA;
            plan->fz_slots[f] = (int64_t)plan->sm_count * std::max(1, bps);
        }
        for (int k = 0; k < plan->conc; ++k) {
            if (!plan->fside[k] && cudaStreamCreateWithFlags(&plan->fside[k], cudaStreamNonBlocking) != cudaSuccess)
                return SWDFT_ERR_CUDA;
            if (!plan->fjoin_ev[k] && cudaEventCreateWithFlags(&plan->fjoin_ev[k], cudaEventDisableTiming) != cudaSuccess)
                return SWDFT_ERR_CUDA;
        }
    }
    plan->configured = true;
    return SWDFT_OK;
}

// Build and upload the pipelined classes' item table (a plan constant; again after autotuning
// changed the arrays' chunks).  Synchronous: not while a stream is capturing.
swdft_status pipe_ready(swdft2d_plan_t plan) {
    if (plan->pipe_uploaded) return SWDFT_OK;
    std::vector<BatchPipeItem> items;
    build_pipe(plan, items, plan->pipe_sync);
    const size_t bytes = sizeof(BatchPipeItem) * std::max<size_t>(1, items.size());
    if (bytes > plan->pipe_dev_bytes) {
        if (plan->pipe_dev) {
            if (cudaDeviceSynchronize() != cudaSuccess) return SWDFT_ERR_CUDA;  // a graph may still read it
            cudaFree(plan->pipe_dev);
            plan->pipe_dev = nullptr;
            plan->pipe_dev_bytes = 0;
        }
        if (alloc_fails() || cudaMalloc((void **)&plan->pipe_dev, bytes) != cudaSuccess) return SWDFT_ERR_OOM;
        plan->pipe_dev_bytes = bytes;
    } else if (cudaDeviceSynchronize() != cudaSuccess) {
        return SWDFT_ERR_CUDA;
    }
    if (!items.empty() &&
        cudaMemcpy(plan->pipe_dev, items.data(), sizeof(BatchPipeItem) * items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return SWDFT_ERR_CUDA;
    plan->pipe_uploaded = true;
    return SWDFT_OK;
}

// Fill the pinned batch descriptors for these buffers.  The caller makes sure no pending
// copy still reads them.
void fill_batch(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out, void *ws) {
    const size_t n = plan->arrays.size();
    BatchImage *imgs = reinterpret_cast<BatchImage *>(plan->desc_host);
    BatchClassEntry *fz_ent = reinterpret_cast<BatchClassEntry *>(imgs + n);
    for (size_t i = 0; i < n; ++i) {
        const ArrayPlan &a = plan->arrays[i];
        BatchImage d;
        std::memset(&d, 0, sizeof(d));
        float2 *z = reinterpret_cast<float2 *>(static_cast<char *>(ws) + plan->z_off[i]) + a.z_pad() * a.P1 * a.n1;
        const int64_t zrows = a.band_rows() + a.n0 - 1;
        d.row.x = static_cast<const char *>(d_in[i]);
        d.row.ld = a.ld;
        d.row.r_base = a.q_begin;
        d.row.zrow = a.P1 * a.n1;
        d.row.rows = (int)zrows;
        d.row.P1 = (int)a.P1;
        d.row.z = z;
        d.col.z = z;
        d.col.out = static_cast<float2 *>(d_out[i]);
        d.col.nch = a.P1 * a.n1;
        d.col.orow = a.P1 * a.n1 * a.n0;
        d.col.rows_out = (int)a.band_rows();
        d.col.m1 = a.m1;
        d.col.groups = batch_col_groups(a.m0);
        d.col.scale = norm_scale(plan->norm, a.n0, a.n1);
        d.m0 = a.m0;
        d.m1 = a.m1;
        d.cplx = a.dtype == SWDFT_C64;
        d.fused = a.batch_mode == kBatchFused ? 1 : 0;
        const int64_t ch_per_block = 32LL * d.col.groups;
        d.col_blocks = (int)((d.col.nch + ch_per_block - 1) / ch_per_block);
        if (a.batch_mode == kBatchFused) {
            d.col.chunk = (int)std::min<int64_t>(a.band_rows(), std::max<int64_t>(1, a.cfg.col_chunk));
            d.col_chunks = (int)((a.band_rows() + d.col.chunk - 1) / d.col.chunk);
        } else {
            const PipeGeom g = pipe_geom(a);
            d.row.chunk = g.row_chunk;
            d.row_blocks = g.row_blocks;
            d.row_chunks = g.row_chunks;
            d.col.chunk = g.col_chunk;
            d.col_chunks = g.col_chunks;
            d.col_blocks = g.col_blocks;
            d.sync_off = plan->pipe_sync[i];
        }
        imgs[i] = d;
    }
    // fused groups: column tiles of the fused arrays, grouped by (m0, m1)
    int pos = 0;
    for (int f = 0; f < swdft2d_plan_s::kFz; ++f) {
        plan->fz_off[f] = pos;
        int64_t items = 0;
        for (size_t i = 0; i < n; ++i)
            if (imgs[i].fused && imgs[i].m0 * kBatchFusedM1 + imgs[i].m1 == f) {
                fz_ent[pos].item0 = items;
                fz_ent[pos].img = (int)i;
                fz_ent[pos].pad = 0;
                items += (int64_t)imgs[i].col_blocks * imgs[i].col_chunks;
                ++pos;
            }
        plan->fz_n[f] = pos - plan->fz_off[f];
        plan->fz_items[f] = items;
    }
}

cudaError_t enqueue_forward(const swdft2d_plan_s *plan, const ArrayPlan &a, const void *in, void *out, void *ws,
                            int64_t q_lo, int64_t q_hi, cudaStream_t s, int stages = 3);

// Zero the pipelined kernels' counters, then run, concurrently on the plan's side streams and
// joined back into s: the pipelined kernel of every window shape with arrays in that mode, the
// fused kernel of every window shape with fused arrays, and the per-array launches of the
// arrays that run on their own.  only >= 0 restricts it all to the arrays of window shape
// `only` (m0 * 7 + m1; the autotuner's timing runs).  Only memsets, event records/waits and
// kernel launches (capturable).
swdft_status launch_batch(swdft2d_plan_t plan, const unsigned char *desc, const void *const *d_in,
                          void *const *d_out, void *ws, cudaStream_t s, int only = -1) {
    const size_t n = plan->arrays.size();
    const BatchImage *imgs = reinterpret_cast<const BatchImage *>(desc);
    const BatchClassEntry *fz_ent = reinterpret_cast<const BatchClassEntry *>(imgs + n);
    swdft_status st = SWDFT_OK;
    int *sync = reinterpret_cast<int *>(static_cast<char *>(ws) + plan->sync_off);
    if (cudaMemsetAsync(sync, 0, plan->sync_bytes, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    if (cudaEventRecord(plan->fork_ev, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    for (int j = 0; j < plan->conc; ++j)
        if (cudaStreamWaitEvent(plan->side[j], plan->fork_ev, 0) != cudaSuccess ||
            cudaStreamWaitEvent(plan->fside[j], plan->fork_ev, 0) != cudaSuccess)
            return SWDFT_ERR_CUDA;
    auto cls = [](const ArrayPlan &a) { return a.m0 * (kMaxLog2 + 1) + a.m1; };
    int k = 0;
    BatchPipeArgs pa;
    pa.imgs = imgs;
    const BatchPipeItem *items = reinterpret_cast<const BatchPipeItem *>(plan->pipe_dev);
    pa.abort = sync + swdft2d_plan_s::kPz;
    pa.done = sync + swdft2d_plan_s::kPipeHead;
    pa.budget = g_pipe_budget.load(std::memory_order_relaxed);
    pa.poison = g_pipe_poison.load(std::memory_order_relaxed);
    pa.om64 = plan->om64;
    for (int c = 0; c < swdft2d_plan_s::kPz && st == SWDFT_OK; ++c) {
        if (plan->pz_n[c] == 0 || (only >= 0 && c != only)) continue;
        pa.items = items + plan->pz_off[c];
        pa.nitems = plan->pz_n[c];
        pa.ticket = sync + c;
        if (launch_batch_pipe(c / (kMaxLog2 + 1), c % (kMaxLog2 + 1), pa, plan->pz_slots[c],
                              plan->side[k++ % plan->conc]) != cudaSuccess)
            st = SWDFT_ERR_CUDA;
    }
    // fused groups need no z: they run beside the pipelined kernels on their own streams
    int kf = 0;
    for (int f = 0; f < swdft2d_plan_s::kFz && st == SWDFT_OK; ++f) {
        const int m0 = f / kBatchFusedM1, m1 = f % kBatchFusedM1;
        if (plan->fz_n[f] == 0 || (only >= 0 && m0 * (kMaxLog2 + 1) + m1 != only)) continue;
        if (launch_batch_fused_class(m0, m1, imgs, fz_ent + plan->fz_off[f], plan->fz_n[f], plan->fz_items[f],
                                     plan->om64, plan->fz_slots[f], plan->fside[kf++ % plan->conc]) != cudaSuccess)
            st = SWDFT_ERR_CUDA;
    }
    // arrays on their own: their per-array launches (tree or tensor-core form) in their region
    for (size_t i = 0; i < n && st == SWDFT_OK; ++i) {
        const ArrayPlan &a = plan->arrays[i];
        if (a.batch_mode != kBatchSolo || (only >= 0 && cls(a) != only)) continue;
        if (enqueue_forward(plan, a, d_in[i], d_out[i], static_cast<char *>(ws) + plan->z_off[i], a.q_begin, a.q_end,
                            plan->side[k++ % plan->conc]) != cudaSuccess)
            st = SWDFT_ERR_CUDA;
    }
    // always join every forked stream back (a capture must end with every stream joined)
    for (int j = 0; j < plan->conc; ++j) {
        if (cudaEventRecord(plan->join_ev[j], plan->side[j]) != cudaSuccess) st = SWDFT_ERR_CUDA;
        if (cudaStreamWaitEvent(s, plan->join_ev[j], 0) != cudaSuccess) st = SWDFT_ERR_CUDA;
        if (cudaEventRecord(plan->fjoin_ev[j], plan->fside[j]) != cudaSuccess) st = SWDFT_ERR_CUDA;
        if (cudaStreamWaitEvent(s, plan->fjoin_ev[j], 0) != cudaSuccess) st = SWDFT_ERR_CUDA;
    }
    return st;
}

// Direct (non-graph) persistent execute: refill the staging once its previous upload ran,
// upload it on the stream and launch the two persistent passes.
swdft_status enqueue_batch(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out,
                           void *ws, cudaStream_t s) {
    swdft_status st = pipe_ready(plan);
    if (st != SWDFT_OK) return st;
    if (cudaEventSynchronize(plan->desc_uploaded) != cudaSuccess) return SWDFT_ERR_CUDA;
    fill_batch(plan, d_in, d_out, ws);
    if (cudaMemcpyAsync(plan->desc_dev, plan->desc_host, plan->desc_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SWDFT_ERR_CUDA;
    if (cudaEventRecord(plan->desc_uploaded, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    return launch_batch(plan, plan->desc_dev, d_in, d_out, ws, s);
}

// Enqueue the forward transform of output rows [q_lo, q_hi) of array a.
// stages: bit 0 = row levels (x -> z), bit 1 = column levels (z -> out).
cudaError_t enqueue_forward(const swdft2d_plan_s *plan, const ArrayPlan &a, const void *in,
                            void *out, void *ws, int64_t q_lo, int64_t q_hi, cudaStream_t s,
                            int stages) {
    const int64_t rows_out = q_hi - q_lo;
    if (rows_out <= 0) return cudaSuccess;
    if (a.algo >= SWDFT_ALGO_TC_BF16X3) {
        // tensor-core form: row DFT (tcgen05) -> operand planes -> column DFT (tcgen05)
        const int terms = ArrayPlan::tc_terms(a.algo);
        const bool f16 = a.algo == SWDFT_ALGO_TC_F16 || a.algo == SWDFT_ALGO_TC_F16_SCALED;
        const bool scaled = a.algo == SWDFT_ALGO_TC_F16_SCALED;
        char *planes = static_cast<char *>(ws);
        float *amax = reinterpret_cast<float *>(planes + align_up(a.planes_bytes(rows_out, a.algo)));
        if (stages & 1) {
            TcRowArgs tr;
            tr.x = static_cast<const char *>(in) + (size_t)q_lo * a.ld * a.in_elem();
            tr.ld = a.ld;
            tr.cplx = a.dtype == SWDFT_C64;
            tr.N1 = a.N1;
            tr.P1 = a.P1;
            tr.zrows = rows_out + a.n0 - 1;
            tr.m1 = a.m1;
            tr.planes = planes;
            tr.terms = terms;
            tr.f16 = f16;
            tr.amax = scaled ? amax : nullptr;
            tr.om64 = plan->om64;
            cudaError_t e = launch_tc_row(tr, s);
            if (e != cudaSuccess) return e;
        }
        if (!(stages & 2)) return cudaSuccess;
        TcColArgs t;
        t.planes = planes;
        t.terms = terms;
        t.f16 = f16;
        t.amax = scaled ? amax : nullptr;
        t.amax_mult = (float)a.n1;
        t.P1 = a.P1;
        t.rows_out = rows_out;
        t.m0 = a.m0;
        t.m1 = a.m1;
        t.out = static_cast<float2 *>(out);
        t.scale = norm_scale(plan->norm, a.n0, a.n1);
        t.om64 = plan->om64;
        t.chunk = a.tc_chunk;
        return launch_tc_col(t, s);
    }
    if (a.ternary()) {
        // ternary trees along one or both axes (tree3.cu): a row pass (ternary, or binary
        // when n1 is a power of two), then the ternary column pass over z rows of any length
        float2 *z = static_cast<float2 *>(ws) + a.z_pad() * a.P1 * a.n1;
        if (stages & 1) {
            cudaError_t e;
            if (a.r1 == 3) {
                Row3Args r;
                r.x = in;
                r.ld = a.ld;
                r.cplx = a.dtype == SWDFT_C64;
                r.r_base = q_lo;
                r.rows = rows_out + a.n0 - 1;
                r.P1 = a.P1;
                r.b1 = a.b1;
                r.a1 = a.a1;
                r.z = z;
                r.chunk = a.cfg.row_chunk;
                e = launch_row_tree3(r, s);
            } else {
                RowTreeArgs r;
                r.x = in;
                r.ld = a.ld;
                r.cplx = a.dtype == SWDFT_C64;
                r.r_base = q_lo;
                r.rows = rows_out + a.n0 - 1;
                r.P1 = a.P1;
                r.m1 = a.m1;
                r.z = z;
                r.om64 = plan->om64;
                r.B = a.cfg.row_B;
                r.chunk = a.cfg.row_chunk;
                e = launch_row_tree(r, s);
            }
            if (e != cudaSuccess) return e;
        }
        if (!(stages & 2)) return cudaSuccess;
        Col3Args c;
        c.z = z;
        c.P1 = a.P1;
        c.rows_out = rows_out;
        c.n1 = a.n1;
        c.b0 = a.b0;  // n0 = 3^b0 2^a0, or n0 = 1
        c.a0 = a.a0;
        c.out = static_cast<float2 *>(out);
        c.scale = norm_scale(plan->norm, a.n0, a.n1);
        c.chunk = a.cfg.col_chunk;
        return launch_col_tree3(c, s);
    }
    if (a.cfg.fused && fused_supported(a.m0, a.m1)) {
        // one launch: row levels inside the column tile; stage 0 has nothing to do
        if (!(stages & 2)) return cudaSuccess;
        FusedTreeArgs f;
        f.x = static_cast<const char *>(in) + (size_t)q_lo * a.ld * a.in_elem();
        f.ld = a.ld;
        f.cplx = a.dtype == SWDFT_C64;
        f.P1 = a.P1;
        f.rows_out = rows_out;
        f.m0 = a.m0;
        f.m1 = a.m1;
        f.out = static_cast<float2 *>(out);
        f.scale = norm_scale(plan->norm, a.n0, a.n1);
        f.om64 = plan->om64;
        f.chunk = a.cfg.col_chunk;
        f.groups = a.cfg.col_groups;
        return launch_fused_tree(f, s);
    }
    RowTreeArgs r;
    r.x = in;
    r.ld = a.ld;
    r.cplx = a.dtype == SWDFT_C64;
    r.r_base = q_lo;
    r.rows = rows_out + a.n0 - 1;
    r.P1 = a.P1;
    r.m1 = a.m1;
    float2 *z = static_cast<float2 *>(ws) + a.z_pad() * a.P1 * a.n1;
    r.z = z;
    r.om64 = plan->om64;
    r.B = a.cfg.row_B;
    r.chunk = a.cfg.row_chunk;
    if (stages & 1) {
        cudaError_t e = launch_row_tree(r, s);
        if (e != cudaSuccess) return e;
    }
    if (!(stages & 2)) return cudaSuccess;
    ColTreeArgs c;
    c.z = z;
    c.P1 = a.P1;
    c.rows_out = rows_out;
    c.m0 = a.m0;
    c.m1 = a.m1;
    c.out = static_cast<float2 *>(out);
    c.scale = norm_scale(plan->norm, a.n0, a.n1);
    c.om64 = plan->om64;
    c.B = a.cfg.col_B;
    c.chunk = a.cfg.col_chunk;
    c.groups = a.cfg.col_groups;
    c.z_full = static_cast<const float2 *>(ws);  // z's padding rows start the workspace
    c.z_pad = a.z_pad();
    return launch_col_tree(c, s);
}

// Run body(i, stream, workspace slot) for every array: on the caller's stream when the plan
// has one array, else forked over the plan's side streams and joined back to s.
template <class Body>
swdft_status for_each_array(swdft2d_plan_t plan, void *ws, cudaStream_t s, Body body) {
    const size_t n = plan->arrays.size();
    if (plan->conc <= 1) {
        for (size_t i = 0; i < n; ++i)
            if (body(i, s, ws) != cudaSuccess) return SWDFT_ERR_CUDA;
        return SWDFT_OK;
    }
    if (cudaEventRecord(plan->fork_ev, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    for (int k = 0; k < plan->conc; ++k)
        if (cudaStreamWaitEvent(plan->side[k], plan->fork_ev, 0) != cudaSuccess) return SWDFT_ERR_CUDA;
    swdft_status st = SWDFT_OK;
    const bool own_region = (plan->flags & SWDFT_FLAG_PERSISTENT) != 0;  // one region per array
    for (size_t i = 0; i < n && st == SWDFT_OK; ++i) {
        const int k = (int)(i % plan->conc);
        void *slot = static_cast<char *>(ws) + (own_region ? plan->z_off[i] : (size_t)k * plan->slot_bytes);
        if (body(i, plan->side[k], slot) != cudaSuccess) st = SWDFT_ERR_CUDA;
    }
    // always join every side stream back (a capture must end with all streams joined)
    for (int k = 0; k < plan->conc; ++k) {
        if (cudaEventRecord(plan->join_ev[k], plan->side[k]) != cudaSuccess) st = SWDFT_ERR_CUDA;
        if (cudaStreamWaitEvent(s, plan->join_ev[k], 0) != cudaSuccess) st = SWDFT_ERR_CUDA;
    }
    return st;
}

swdft_status enqueue_all(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out,
                         void *ws, cudaStream_t s, int stages = 3) {
    return for_each_array(plan, ws, s, [&](size_t i, cudaStream_t st, void *slot) {
        const ArrayPlan &a = plan->arrays[i];
        return enqueue_forward(plan, a, d_in[i], d_out[i], slot, a.q_begin, a.q_end, st, stages);
    });
}

swdft_status check_buffers(swdft2d_plan_t plan, const void *const *in, void *const *out,
                           void *ws) {
    if (!in || !out) return SWDFT_ERR_INVALID_ARG;
    for (size_t i = 0; i < plan->arrays.size(); ++i) {
        const ArrayPlan &a = plan->arrays[i];
        if (!in[i] || !out[i]) return SWDFT_ERR_INVALID_ARG;
        if ((uintptr_t)in[i] % a.in_elem() != 0) return SWDFT_ERR_INVALID_ARG;
        if ((uintptr_t)out[i] % 16 != 0) return SWDFT_ERR_INVALID_ARG;
    }
    if (plan->ws_bytes > 0 && (!ws || (uintptr_t)ws % kAlign != 0)) return SWDFT_ERR_WORKSPACE;
    return SWDFT_OK;
}

void destroy_graph(GraphCache &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
    g.stream = nullptr;
}

// The autotuner's record of one array: one JSON object per line of the tuning cache, read
// back by swdft2d_load_tuning with the same layout (GPU name, array, choice, time).
#define SWDFT_TUNE_FIELDS(GPU, MS)                                                                \
    "{\"gpu\": \"" GPU "\", \"N0\": %lld, \"N1\": %lld, \"ld\": %lld, \"n0\": %d, \"n1\": %d, "        \
    "\"dtype\": %d, \"q_begin\": %lld, \"q_end\": %lld, \"auto\": %d, \"algo\": %d, \"fused\": %d, "   \
    "\"row_B\": %d, \"row_chunk\": %lld, \"col_B\": %d, \"col_chunk\": %lld, \"col_groups\": %d, "     \
    "\"ms\": " MS "}"

struct TuneRecord {
    char gpu[128];
    long long N0, N1, ld, q_begin, q_end, row_chunk, col_chunk;
    int n0, n1, dtype, autoflag, algo, fused, row_B, col_B, col_groups;
    double ms;
};

bool parse_tune_record(const char *line, TuneRecord *r) {
    const int got = std::sscanf(line, SWDFT_TUNE_FIELDS("%127[^\"]", "%lf"), r->gpu, &r->N0, &r->N1, &r->ld,
                                &r->n0, &r->n1, &r->dtype, &r->q_begin, &r->q_end, &r->autoflag, &r->algo,
                                &r->fused, &r->row_B, &r->row_chunk, &r->col_B, &r->col_chunk, &r->col_groups,
                                &r->ms);
    return got == 18;
}

void write_tune_record(FILE *f, const char *gpu, const ArrayPlan &a, const TreeConfig &c, double ms) {
    std::fprintf(f, SWDFT_TUNE_FIELDS("%s", "%.6f") "\n", gpu, (long long)a.N0, (long long)a.N1, (long long)a.ld,
                 a.n0, a.n1, a.dtype, (long long)a.q_begin, (long long)a.q_end, a.algo_auto ? 1 : 0, a.algo,
                 c.fused ? 1 : 0, c.row_B, (long long)c.row_chunk, c.col_B, (long long)c.col_chunk, c.col_groups,
                 ms);
}

// A record for this array (same GPU, shape, row stride, band, dtype and algorithm setting)
// whose choice is one the plan can run: its configuration and algorithm.
bool tune_record_applies(const TuneRecord &r, const char *gpu, const ArrayPlan &a, TreeConfig *c, int *algo) {
    if (std::strcmp(r.gpu, gpu) != 0 || r.N0 != a.N0 || r.N1 != a.N1 || r.ld != a.ld || r.n0 != a.n0 ||
        r.n1 != a.n1 || r.dtype != a.dtype || r.q_begin != a.q_begin || r.q_end != a.q_end ||
        (r.autoflag != 0) != a.algo_auto || a.ternary())
        return false;
    if (a.algo_auto ? !(r.algo == SWDFT_ALGO_TREE_F32 || (r.algo == SWDFT_ALGO_TC_BF16X3 && a.tc_eligible()))
                    : r.algo != a.algo)
        return false;
    if (r.row_B < 0 || r.row_B > std::min(a.m1, 3) || r.col_B < 0 || r.col_B > std::min(a.m0, 3) ||
        r.row_chunk < 0 || r.col_chunk < 0 || r.col_groups < 1 || r.col_groups > 8 || r.fused < 0 || r.fused > 1 ||
        (r.fused == 1 && !fused_supported(a.m0, a.m1)))
        return false;
    // chunks so short that a pass would need more than 65535 of them (the grid's y limit) on
    // this array's band: a stale or hand-edited record, not one the autotuner writes
    const auto too_many = [](int64_t extent, long long chunk) {
        return chunk > 0 && (extent + chunk - 1) / chunk > 65535;
    };
    if (too_many(a.P1, r.row_chunk) || too_many(a.band_rows(), r.col_chunk)) return false;
    c->fused = r.fused == 1;
    c->row_B = r.row_B;
    c->row_chunk = r.row_chunk;
    c->col_B = r.col_B;
    c->col_chunk = r.col_chunk;
    c->col_groups = r.col_groups;
    *algo = r.algo;
    return true;
}

// Apply the last applicable record of `path` to every array; loaded[i] = 1 for those set.
int load_tuning(swdft2d_plan_t plan, const char *path, const char *gpu, std::vector<char> &loaded) {
    loaded.assign(plan->arrays.size(), 0);
    FILE *f = std::fopen(path, "r");
    if (!f) return 0;
    std::vector<TreeConfig> cfg(plan->arrays.size());
    std::vector<int> algo(plan->arrays.size(), 0);
    char line[1024];
    TuneRecord r;
    while (std::fgets(line, sizeof line, f)) {
        if (!parse_tune_record(line, &r)) continue;
        for (size_t i = 0; i < plan->arrays.size(); ++i)
            if (tune_record_applies(r, gpu, plan->arrays[i], &cfg[i], &algo[i])) loaded[i] = 1;
    }
    std::fclose(f);
    int n = 0;
    for (size_t i = 0; i < plan->arrays.size(); ++i) {
        if (!loaded[i]) continue;
        ArrayPlan &a = plan->arrays[i];
        a.cfg = cfg[i];
        a.algo = algo[i];
        a.tuned = true;
        ++n;
    }
    if (n > 0) destroy_graph(plan->graph);
    return n;
}

bool device_name(char *buf, size_t len) {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
    std::snprintf(buf, len, "%s", prop.name);
    return true;
}

}  // namespace

extern "C" {

int32_t swdft2d_version(void) { return 200; }  // 0.2.0: tuning cache read-back, failure test hooks

const char *swdft2d_status_string(int32_t s) {
    switch (s) {
        case SWDFT_OK: return "SWDFT_OK";
        case SWDFT_ERR_INVALID_ARG: return "SWDFT_ERR_INVALID_ARG: invalid argument";
        case SWDFT_ERR_NOT_POW2: return "SWDFT_ERR_NOT_POW2: window sides must be powers of two or of three";
        case SWDFT_ERR_WINDOW_TOO_LARGE: return "SWDFT_ERR_WINDOW_TOO_LARGE: window larger than the array";
        case SWDFT_ERR_UNSUPPORTED: return "SWDFT_ERR_UNSUPPORTED: not implemented for this request";
        case SWDFT_ERR_OOM: return "SWDFT_ERR_OOM: allocation failed";
        case SWDFT_ERR_CUDA: return "SWDFT_ERR_CUDA: a CUDA call failed";
        case SWDFT_ERR_DEVICE_TIMEOUT: return "SWDFT_ERR_DEVICE_TIMEOUT: a bounded device wait ran out";
        case SWDFT_ERR_WORKSPACE: return "SWDFT_ERR_WORKSPACE: workspace missing or misaligned";
        default: return "unknown swdft status";
    }
}

swdft_status swdft2d_plan(swdft2d_plan_t *out, int32_t batch, const swdft2d_shape *shapes,
                          int32_t norm, int32_t pos, int32_t algo, uint32_t flags) {
    if (!out) return SWDFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (batch < 1 || !shapes) return SWDFT_ERR_INVALID_ARG;
    if (norm < SWDFT_NORM_UNITARY || norm > SWDFT_NORM_INV_N) return SWDFT_ERR_INVALID_ARG;
    if (pos != SWDFT_POS_START && pos != SWDFT_POS_END) return SWDFT_ERR_INVALID_ARG;
    if (algo < SWDFT_ALGO_AUTO || algo > SWDFT_ALGO_TC_F16) return SWDFT_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)(SWDFT_FLAG_GRAPH | SWDFT_FLAG_HOST_IO | SWDFT_FLAG_PERSISTENT | SWDFT_FLAG_AUTOTUNE))
        return SWDFT_ERR_INVALID_ARG;

    std::vector<ArrayPlan> arrays((size_t)batch);
    for (int32_t i = 0; i < batch; ++i) {
        const swdft2d_shape &s = shapes[i];
        ArrayPlan &a = arrays[(size_t)i];
        if (s.N0 < 1 || s.N1 < 1 || s.n0 < 1 || s.n1 < 1) return SWDFT_ERR_INVALID_ARG;
        if (s.dtype != SWDFT_R32 && s.dtype != SWDFT_C64) return SWDFT_ERR_INVALID_ARG;
        int m0 = log2_exact(s.n0), m1 = log2_exact(s.n1), r0 = 2, r1 = 2, b0 = 0, a0 = 0, b1 = 0, a1 = 0;
        if (m0 < 0 && mixed_split(s.n0, &b0, &a0)) {
            r0 = 3;
            m0 = b0;
        }
        if (m1 < 0 && mixed_split(s.n1, &b1, &a1)) {
            r1 = 3;
            m1 = b1;
        }
        if (m0 < 0 || m1 < 0) return SWDFT_ERR_NOT_POW2;
        if (s.n0 > s.N0 || s.n1 > s.N1) return SWDFT_ERR_WINDOW_TOO_LARGE;
        const int64_t ld = s.ld == 0 ? s.N1 : s.ld;
        if (ld < s.N1) return SWDFT_ERR_INVALID_ARG;
        a.N0 = s.N0;
        a.N1 = s.N1;
        a.ld = ld;
        a.n0 = s.n0;
        a.n1 = s.n1;
        a.m0 = m0;
        a.m1 = m1;
        a.r0 = r0;
        a.r1 = r1;
        a.b0 = b0;
        a.a0 = a0;
        a.b1 = b1;
        a.a1 = a1;
        a.dtype = s.dtype;
        a.P0 = s.N0 - s.n0 + 1;
        a.P1 = s.N1 - s.n1 + 1;
        // band of window rows in q coordinates
        const int64_t shift = (pos == SWDFT_POS_END) ? (s.n0 - 1) : 0;
        int64_t b = s.row_begin, e = s.row_end;
        if (e == 0 && b == 0) {
            a.q_begin = 0;
            a.q_end = a.P0;
        } else {
            if (e == 0) e = a.P0 + shift;
            a.q_begin = b - shift;
            a.q_end = e - shift;
            if (a.q_begin < 0 || a.q_end > a.P0 || a.q_begin >= a.q_end) return SWDFT_ERR_INVALID_ARG;
        }
        // trees built: 2^m <= 64; 3^b 2^a <= 64 (b <= 3)
        if ((r0 == 3 ? (s.n0 > kMaxN || b0 > kMaxLog3) : m0 > kMaxLog2) ||
            (r1 == 3 ? (s.n1 > kMaxN || b1 > kMaxLog3) : m1 > kMaxLog2))
            return SWDFT_ERR_UNSUPPORTED;
        // a ternary row tree feeds the ternary column kernel (z rows of any length); the
        // binary column kernel needs power-of-two rows
        if (r1 == 3 && r0 == 2 && m0 > 0) return SWDFT_ERR_UNSUPPORTED;
        a.algo = (algo == SWDFT_ALGO_AUTO) ? SWDFT_ALGO_TREE_F32 : algo;
        a.algo_auto = algo == SWDFT_ALGO_AUTO;
        if (a.algo >= SWDFT_ALGO_TC_BF16X3 && !a.tc_eligible()) return SWDFT_ERR_UNSUPPORTED;
    }

    swdft2d_plan_s *p = alloc_fails() ? nullptr : new (std::nothrow) swdft2d_plan_s();
    if (!p) return SWDFT_ERR_OOM;
    p->arrays = std::move(arrays);
    p->norm = norm;
    p->pos = pos;
    p->algo = (algo == SWDFT_ALGO_AUTO) ? SWDFT_ALGO_TREE_F32 : algo;
    p->flags = flags;
    make_omega(kMaxN, p->om64);
    size_t ws = 0;
    if (flags & SWDFT_FLAG_PERSISTENT) {
        // the batch's kernels run at once, so each array has its own region (its z, or the
        // tensor-core form's operand planes when that form may run); the kernels run on up to
        // four side streams
        for (const auto &a : p->arrays) {
            p->z_off.push_back(ws);
            ws += align_up(a.ws_bytes_plan(a.band_rows()));
        }
        p->conc = 4;
        // tensor-core forms and ternary or mixed-radix windows run per array beside the
        // persistent kernels; small windows (n0 n1 <= 64, where z is 1/n0 >= 1/8 of the
        // output) in fused groups; every other array in the pipelined kernel of its (n0, n1).
        // The autotuner may move radix-2 tree arrays between the three, per window shape.
        // Every array has row-tile flags, whatever its mode.
        for (auto &a : p->arrays) {
            a.batch_mode = (a.algo >= SWDFT_ALGO_TC_BF16X3 || a.ternary()) ? kBatchSolo
                           : (a.m1 < kBatchFusedM1 && a.n0 * a.n1 <= 64) ? kBatchFused
                                                                          : kBatchPipe;
            const PipeGeom g = pipe_geom(a);
            p->pipe_flags += g.row_blocks * g.row_chunks;
        }
        p->sync_off = ws;
        p->sync_bytes = sizeof(int) * ((size_t)swdft2d_plan_s::kPipeHead + (size_t)p->pipe_flags);
        ws += align_up(p->sync_bytes);
    } else {
        // up to four arrays run at once (plan-owned streams), each with its own z slot;
        // arrays of one shape run their adjoint passes in groups of up to kAdjZ launches
        const ArrayPlan &f = p->arrays.front();
        p->uniform = p->arrays.size() > 1;
        for (const auto &a : p->arrays)
            p->uniform = p->uniform && a.N0 == f.N0 && a.N1 == f.N1 && a.ld == f.ld && a.n0 == f.n0 &&
                         a.n1 == f.n1 && a.dtype == f.dtype && a.q_begin == f.q_begin && a.q_end == f.q_end &&
                         !a.ternary();
        for (const auto &a : p->arrays) ws = std::max(ws, align_up(a.ws_bytes_plan(a.band_rows())));
        p->conc = (int)std::min<size_t>(kConc, p->arrays.size());
        p->slot_bytes = ws;
        const size_t slots = p->uniform ? std::max<size_t>((size_t)p->conc, std::min<size_t>(kAdjZ, p->arrays.size()))
                                        : (size_t)p->conc;
        ws *= slots;
    }
    p->ws_bytes = ws;
    // launch shapes known at plan time (so launch_count is right before the first execute)
    for (auto &a : p->arrays) default_config(a, p->sm_count, p->conc);
    *out = p;
    return SWDFT_OK;
}

swdft_status swdft2d_output_shape(swdft2d_plan_t plan, int32_t i, int64_t out[4]) {
    if (!plan || !out || i < 0 || (size_t)i >= plan->arrays.size()) return SWDFT_ERR_INVALID_ARG;
    const ArrayPlan &a = plan->arrays[(size_t)i];
    out[0] = a.band_rows();
    out[1] = a.P1;
    out[2] = a.n0;
    out[3] = a.n1;
    return SWDFT_OK;
}

swdft_status swdft2d_workspace_size(swdft2d_plan_t plan, size_t *bytes) {
    if (!plan || !bytes) return SWDFT_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return SWDFT_OK;
}

swdft_status swdft2d_get_algo(swdft2d_plan_t plan, int32_t *algo) {
    if (!plan || !algo) return SWDFT_ERR_INVALID_ARG;
    *algo = plan->arrays.front().algo;  // after autotuning, the form array 0 runs
    return SWDFT_OK;
}

swdft_status swdft2d_get_form(swdft2d_plan_t plan, int32_t i, int32_t *algo, int32_t *form) {
    if (!plan || i < 0 || (size_t)i >= plan->arrays.size()) return SWDFT_ERR_INVALID_ARG;
    const ArrayPlan &a = plan->arrays[(size_t)i];
    static_assert(kBatchPipe == SWDFT_FORM_PIPELINED && kBatchFused == SWDFT_FORM_FUSED_GROUP &&
                      kBatchSolo == SWDFT_FORM_PER_ARRAY,
                  "batch modes are the public forms");
    if (algo) *algo = a.algo;
    if (form) *form = (plan->flags & SWDFT_FLAG_PERSISTENT) ? a.batch_mode : SWDFT_FORM_PER_ARRAY;
    return SWDFT_OK;
}

swdft_status swdft2d_launch_count(swdft2d_plan_t plan, int32_t adjoint, int32_t *launches) {
    if (!plan || !launches) return SWDFT_ERR_INVALID_ARG;
    // forward: row + column pass per array, or the two persistent passes for the whole batch;
    // adjoint: column + row adjoint pass per array
    if (!adjoint && (plan->flags & SWDFT_FLAG_PERSISTENT)) {
        // one pipelined kernel per (n0, n1) of the pipelined arrays, one fused kernel per
        // (n0, n1) of the fused arrays, and the per-array launches of the arrays on their own
        bool c[swdft2d_plan_s::kPz] = {}, f[swdft2d_plan_s::kFz] = {};
        int32_t k = 0;
        for (const auto &a : plan->arrays) {
            if (a.batch_mode == kBatchFused)
                f[a.m0 * kBatchFusedM1 + a.m1] = true;
            else if (a.batch_mode == kBatchPipe)
                c[a.m0 * (kMaxLog2 + 1) + a.m1] = true;
            else
                k += (a.algo == SWDFT_ALGO_TREE_F32 && a.cfg.fused && fused_supported(a.m0, a.m1)) ? 1 : 2;
        }
        for (int j = 0; j < swdft2d_plan_s::kPz; ++j) k += (int)c[j];
        for (int j = 0; j < swdft2d_plan_s::kFz; ++j) k += (int)f[j];
        *launches = k;
        return SWDFT_OK;
    }
    // (the column adjoint adds a second launch when its chunks share rows)
    if (adjoint && plan->uniform) {
        // one launch pair (or three) per group of up to kAdjZ arrays of the same shape
        const ArrayPlan &a = plan->arrays.front();
        const int per = 1 + adj_col_launches(a.band_rows(), a.m0, a.adj_chunk(a.band_rows()));
        *launches = (int32_t)(per * ((plan->arrays.size() + kAdjZ - 1) / kAdjZ));
        return SWDFT_OK;
    }
    int32_t n = 0;
    for (const auto &a : plan->arrays)
        n += adjoint ? (a.ternary() ? 2 : 1 + adj_col_launches(a.band_rows(), a.m0, a.adj_chunk(a.band_rows())))
                     : ((a.algo == SWDFT_ALGO_TREE_F32 && a.cfg.fused && fused_supported(a.m0, a.m1)) ? 1 : 2);
    *launches = n;
    return SWDFT_OK;
}

swdft_status swdft2d_execute(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out,
                             void *d_workspace, void *stream) {
    if (!plan) return SWDFT_ERR_INVALID_ARG;
    swdft_status st = check_buffers(plan, d_in, d_out, d_workspace);
    if (st != SWDFT_OK) return st;
    if ((st = configure(plan)) != SWDFT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((plan->flags & SWDFT_FLAG_AUTOTUNE) && !plan->autotuned) {
        // tune on this execute's buffers first (the timing runs synchronise, so not while the
        // stream is being captured into a graph)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return SWDFT_ERR_CUDA;
        if (cs == cudaStreamCaptureStatusNone) {
            if ((st = swdft2d_autotune(plan, d_in, d_out, d_workspace, stream)) != SWDFT_OK) return st;
            plan->autotuned = true;
        }
    }
    const bool persistent = (plan->flags & SWDFT_FLAG_PERSISTENT) != 0;
    if (!(plan->flags & SWDFT_FLAG_GRAPH) || s == nullptr)
        return persistent ? enqueue_batch(plan, d_in, d_out, d_workspace, s)
                          : enqueue_all(plan, d_in, d_out, d_workspace, s);
    // inside a graph only kernel launches are recorded; a persistent plan's descriptors for
    // these buffers go to the graph's own device buffer before capture
    auto enqueue = [&]() {
        if (!persistent) return enqueue_all(plan, d_in, d_out, d_workspace, s);
        return launch_batch(plan, plan->desc_graph, d_in, d_out, d_workspace, s);
    };

    // CUDA graph: capture the launch sequence once per (buffers, stream), replay after.
    std::vector<const void *> key;
    for (size_t i = 0; i < plan->arrays.size(); ++i) {
        key.push_back(d_in[i]);
        key.push_back(d_out[i]);
    }
    key.push_back(d_workspace);
    GraphCache &g = plan->graph;
    if (!g.exec || g.key != key || g.stream != s) {
        destroy_graph(g);
        if (persistent) {
            // an earlier graph of this plan may still be reading the descriptors on any
            // stream: re-capture is rare, so wait for the whole device
            if (cudaDeviceSynchronize() != cudaSuccess) return SWDFT_ERR_CUDA;
            if ((st = pipe_ready(plan)) != SWDFT_OK) return st;
            fill_batch(plan, d_in, d_out, d_workspace);
            if (cudaMemcpy(plan->desc_graph, plan->desc_host, plan->desc_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
                return SWDFT_ERR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SWDFT_ERR_CUDA;
        swdft_status est = enqueue();
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (est != SWDFT_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return est != SWDFT_OK ? est : SWDFT_ERR_CUDA;
        }
        ce = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            g.exec = nullptr;
            return SWDFT_ERR_CUDA;
        }
        g.key = key;
        g.stream = s;
    }
    return cudaGraphLaunch(g.exec, s) == cudaSuccess ? SWDFT_OK : SWDFT_ERR_CUDA;
}

swdft_status swdft2d_execute_stage(swdft2d_plan_t plan, int32_t stage, const void *const *d_in,
                                   void *const *d_out, void *d_workspace, void *stream) {
    if (!plan || (stage != 0 && stage != 1)) return SWDFT_ERR_INVALID_ARG;
    swdft_status st = check_buffers(plan, d_in, d_out, d_workspace);
    if (st != SWDFT_OK) return st;
    if ((st = configure(plan)) != SWDFT_OK) return st;
    return enqueue_all(plan, d_in, d_out, d_workspace, static_cast<cudaStream_t>(stream), stage == 0 ? 1 : 2);
}

swdft_status swdft2d_set_tree_config(swdft2d_plan_t plan, int32_t i, int32_t row_B,
                                     int64_t row_chunk, int32_t col_B, int64_t col_chunk,
                                     int32_t col_groups, int32_t fused) {
    if (!plan || i < 0 || (size_t)i >= plan->arrays.size()) return SWDFT_ERR_INVALID_ARG;
    if (row_chunk < 0 || col_chunk < 0 || col_groups < 0 || fused < -1 || fused > 1) return SWDFT_ERR_INVALID_ARG;
    ArrayPlan &a = plan->arrays[(size_t)i];
    if (a.ternary() && fused == 1) return SWDFT_ERR_UNSUPPORTED;
    TreeConfig c;
    if (fused == -1) {
        ArrayPlan tmp = a;
        default_config(tmp, plan->sm_count, plan->conc);
        c.fused = tmp.cfg.fused;
    } else {
        c.fused = fused == 1 && fused_supported(a.m0, a.m1) && !a.ternary();
    }
    c.row_B = std::max(0, std::min(row_B, std::min(a.m1, 3)));
    c.row_chunk = row_chunk;
    c.col_B = std::max(0, std::min(col_B, std::min(a.m0, 3)));
    c.col_chunk = col_chunk;
    c.col_groups = std::max(1, col_groups);
    a.cfg = c;
    a.tuned = true;
    destroy_graph(plan->graph);
    return SWDFT_OK;
}

swdft_status swdft2d_execute_adjoint(swdft2d_plan_t plan, const void *const *d_grad_out,
                                     void *const *d_grad_in, void *d_workspace, void *stream) {
    if (!plan || !d_grad_out || !d_grad_in) return SWDFT_ERR_INVALID_ARG;
    for (size_t i = 0; i < plan->arrays.size(); ++i) {
        const ArrayPlan &a = plan->arrays[i];
        if (!d_grad_out[i] || !d_grad_in[i]) return SWDFT_ERR_INVALID_ARG;
        if ((uintptr_t)d_grad_out[i] % sizeof(float2) != 0) return SWDFT_ERR_INVALID_ARG;
        if ((uintptr_t)d_grad_in[i] % a.in_elem() != 0) return SWDFT_ERR_INVALID_ARG;
    }
    if (plan->ws_bytes > 0 && (!d_workspace || (uintptr_t)d_workspace % kAlign != 0)) return SWDFT_ERR_WORKSPACE;
    swdft_status st = configure(plan);
    if (st != SWDFT_OK) return st;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    // ternary and mixed-radix windows: dense per-window inverse DFTs overlap-added per axis
    // (adjoint3.cu), the transposed radix-2 tree for a power-of-two row window
    auto enqueue_mixed = [&](const ArrayPlan &a, const void *G, void *gx_all, void *slot,
                             cudaStream_t s) -> cudaError_t {
        const int64_t zrows = a.band_rows() + a.n0 - 1;
        const size_t row_bytes = (size_t)a.N1 * a.in_elem();
        char *gx = static_cast<char *>(gx_all);
        cudaError_t e;
        if (a.q_begin > 0 && (e = cudaMemsetAsync(gx, 0, (size_t)a.q_begin * row_bytes, s)) != cudaSuccess) return e;
        const int64_t tail = a.N0 - (a.q_begin + zrows);
        if (tail > 0 &&
            (e = cudaMemsetAsync(gx + (size_t)(a.q_begin + zrows) * row_bytes, 0, (size_t)tail * row_bytes, s)) !=
                cudaSuccess)
            return e;
        Adj3ColArgs c;
        c.G = static_cast<const float2 *>(G);
        c.gz = static_cast<float2 *>(slot);
        c.P1 = a.P1;
        c.rows_out = a.band_rows();
        c.n0 = a.n0;
        c.n1 = a.n1;
        c.scale = norm_scale(plan->norm, a.n0, a.n1);
        if ((e = launch_adj3_col(c, s)) != cudaSuccess) return e;
        if (a.r1 == 3) {
            Adj3RowArgs r;
            r.gz = c.gz;
            r.gx = gx + (size_t)a.q_begin * row_bytes;
            r.ld_out = a.N1;
            r.zrows = zrows;
            r.N1 = a.N1;
            r.n1 = a.n1;
            r.cplx = a.dtype == SWDFT_C64;
            return launch_adj3_row(r, s);
        }
        AdjRowArgs r;
        r.gz[0] = c.gz;
        r.gx[0] = gx + (size_t)a.q_begin * row_bytes;
        r.nz = 1;
        r.ld_out = a.N1;
        r.cplx = a.dtype == SWDFT_C64;
        r.zrows = zrows;
        r.N1 = a.N1;
        r.m1 = a.m1;
        r.om64 = plan->om64;
        r.B = 0;
        r.chunk = 0;
        r.sm_count = plan->sm_count;
        return launch_adj_row(r, s);
    };
    // arrays first..first+nz-1 (one shape) in one launch pair; array k of the group uses slots[k]
    auto enqueue_group = [&](size_t first, int nz, void *const *slots, cudaStream_t s) -> cudaError_t {
        const ArrayPlan &a = plan->arrays[first];
        if (a.ternary()) return enqueue_mixed(a, d_grad_out[first], d_grad_in[first], slots[0], s);
        const int64_t zrows = a.band_rows() + a.n0 - 1;
        const size_t row_bytes = (size_t)a.N1 * a.in_elem();
        AdjColArgs c;
        AdjRowArgs r;
        cudaError_t e;
        for (int k = 0; k < nz; ++k) {
            char *gx = static_cast<char *>(d_grad_in[first + k]);
            // rows no window of the band touches get a zero gradient
            if (a.q_begin > 0 && (e = cudaMemsetAsync(gx, 0, (size_t)a.q_begin * row_bytes, s)) != cudaSuccess)
                return e;
            const int64_t tail = a.N0 - (a.q_begin + zrows);
            if (tail > 0 && (e = cudaMemsetAsync(gx + (size_t)(a.q_begin + zrows) * row_bytes, 0,
                                                 (size_t)tail * row_bytes, s)) != cudaSuccess)
                return e;
            c.G[k] = static_cast<const float2 *>(d_grad_out[first + k]);
            c.gz[k] = static_cast<float2 *>(slots[k]);
            c.side[k] = a.adj_side_bytes(a.band_rows()) > 0
                            ? reinterpret_cast<float2 *>(static_cast<char *>(slots[k]) + align_up(a.z_bytes(a.band_rows())))
                            : nullptr;
            r.gz[k] = c.gz[k];
            r.gx[k] = gx + (size_t)a.q_begin * row_bytes;
        }
        c.nz = nz;
        c.P1 = a.P1;
        c.rows_out = a.band_rows();
        c.m0 = a.m0;
        c.m1 = a.m1;
        c.scale = norm_scale(plan->norm, a.n0, a.n1);
        c.om64 = plan->om64;
        c.B = 0;  // the launcher uses the one split built per window side
        c.chunk = a.adj_chunk(a.band_rows());
        if ((e = launch_adj_col(c, s)) != cudaSuccess) return e;
        r.nz = nz;
        r.ld_out = a.N1;
        r.cplx = a.dtype == SWDFT_C64;
        r.zrows = zrows;
        r.N1 = a.N1;
        r.m1 = a.m1;
        r.om64 = plan->om64;
        r.B = 0;  // the launcher uses the one split built per window side
        r.chunk = 0;  // the launcher fills one wave of resident blocks
        r.sm_count = plan->sm_count;
        return launch_adj_row(r, s);
    };
    if (plan->uniform) {
        // one launch pair per group of up to kAdjZ arrays, on the caller's stream
        const size_t n = plan->arrays.size();
        for (size_t first = 0; first < n; first += kAdjZ) {
            const int nz = (int)std::min<size_t>(kAdjZ, n - first);
            void *slots[kAdjZ];
            for (int k = 0; k < nz; ++k) slots[k] = static_cast<char *>(d_workspace) + (size_t)k * plan->slot_bytes;
            if (enqueue_group(first, nz, slots, s0) != cudaSuccess) return SWDFT_ERR_CUDA;
        }
        return SWDFT_OK;
    }
    return for_each_array(plan, d_workspace, s0, [&](size_t i, cudaStream_t s, void *slot) -> cudaError_t {
        void *slots[1] = {slot};
        return enqueue_group(i, 1, slots, s);
    });
}

swdft_status swdft2d_execute_host(swdft2d_plan_t plan, const void *const *h_in,
                                  void *const *h_out, void *stream) {
    if (!plan || !h_in || !h_out) return SWDFT_ERR_INVALID_ARG;
    if (!(plan->flags & SWDFT_FLAG_HOST_IO)) return SWDFT_ERR_INVALID_ARG;
    for (size_t i = 0; i < plan->arrays.size(); ++i)
        if (!h_in[i] || !h_out[i]) return SWDFT_ERR_INVALID_ARG;
    swdft_status st = configure(plan);
    if (st != SWDFT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!plan->io_ready) {
        // band: about 128 MiB of output per slot
        size_t in_max = 0, out_max = 0, ws_max = 0;
        int64_t band = INT64_MAX;
        for (const auto &a : plan->arrays) {
            const int64_t rows = std::max<int64_t>(1, (int64_t)((128u << 20) / a.out_row_bytes()));
            band = std::min(band, rows);
        }
        for (const auto &a : plan->arrays) {
            const int64_t br = std::min(band, a.band_rows());
            in_max = std::max(in_max, align_up((size_t)a.N0 * a.ld * a.in_elem()));
            out_max = std::max(out_max, align_up((size_t)br * a.out_row_bytes()));
            ws_max = std::max(ws_max, align_up(a.ws_bytes_plan(br)));
        }
        // created once, as in configure: a failed attempt keeps what it made for the next
        if (!plan->io_in && (alloc_fails() || cudaMalloc(&plan->io_in, in_max) != cudaSuccess)) return SWDFT_ERR_OOM;
        if (!plan->io_ws && (alloc_fails() || cudaMalloc(&plan->io_ws, ws_max) != cudaSuccess)) return SWDFT_ERR_OOM;
        for (int k = 0; k < 2; ++k)
            if (!plan->io_out[k] && (alloc_fails() || cudaMalloc(&plan->io_out[k], out_max) != cudaSuccess))
                return SWDFT_ERR_OOM;
        if (!plan->io_copy && cudaStreamCreateWithFlags(&plan->io_copy, cudaStreamNonBlocking) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        for (int k = 0; k < 2; ++k) {
            if (!plan->io_done[k] && cudaEventCreateWithFlags(&plan->io_done[k], cudaEventDisableTiming) != cudaSuccess)
                return SWDFT_ERR_CUDA;
            if (!plan->io_copied[k] && cudaEventCreateWithFlags(&plan->io_copied[k], cudaEventDisableTiming) != cudaSuccess)
                return SWDFT_ERR_CUDA;
        }
        plan->io_band = band;
        plan->io_ready = true;
    }
    int64_t slot_uses = 0;
    for (size_t i = 0; i < plan->arrays.size(); ++i) {
        const ArrayPlan &a = plan->arrays[i];
        const size_t in_bytes = (size_t)a.N0 * a.ld * a.in_elem();
        // the input buffer is reused by the next array only after this array's kernels ran
        if (cudaMemcpyAsync(plan->io_in, h_in[i], in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        for (int64_t q = a.q_begin; q < a.q_end; q += plan->io_band) {
            const int64_t qe = std::min(a.q_end, q + plan->io_band);
            const int k = (int)(slot_uses & 1);
            if (slot_uses >= 2 && cudaStreamWaitEvent(s, plan->io_copied[k], 0) != cudaSuccess) return SWDFT_ERR_CUDA;
            if (enqueue_forward(plan, a, plan->io_in, plan->io_out[k], plan->io_ws, q, qe, s) != cudaSuccess)
                return SWDFT_ERR_CUDA;
            if (cudaEventRecord(plan->io_done[k], s) != cudaSuccess) return SWDFT_ERR_CUDA;
            if (cudaStreamWaitEvent(plan->io_copy, plan->io_done[k], 0) != cudaSuccess) return SWDFT_ERR_CUDA;
            char *dst = static_cast<char *>(h_out[i]) + (size_t)(q - a.q_begin) * a.out_row_bytes();
            if (cudaMemcpyAsync(dst, plan->io_out[k], (size_t)(qe - q) * a.out_row_bytes(),
                                cudaMemcpyDeviceToHost, plan->io_copy) != cudaSuccess)
                return SWDFT_ERR_CUDA;
            if (cudaEventRecord(plan->io_copied[k], plan->io_copy) != cudaSuccess) return SWDFT_ERR_CUDA;
            ++slot_uses;
        }
    }
    if (cudaStreamSynchronize(plan->io_copy) != cudaSuccess) return SWDFT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SWDFT_ERR_CUDA;
    return SWDFT_OK;
}

namespace {

// Persistent plans, after the per-array tuning: per window shape (n0, n1), time its arrays in
// each form they may take -- the pipelined kernel, the fused kernel (n1 <= 32), and their own
// launches as just tuned (launch shapes, two-pass or fused, tree or split-bf16) -- each alone
// (launch_batch restricted to that shape, best of three), and keep the fastest.  Arrays made
// with a tensor-core algorithm stay on their own.  Synchronous.
swdft_status autotune_batch(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out, void *ws,
                            cudaStream_t s) {
    const size_t n = plan->arrays.size();
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SWDFT_ERR_CUDA;
    auto cls = [](const ArrayPlan &a) { return a.m0 * (kMaxLog2 + 1) + a.m1; };
    std::vector<int> own_algo(n);  // the per-array tuner's choice
    for (size_t i = 0; i < n; ++i) own_algo[i] = plan->arrays[i].algo;
    auto set_form = [&](int c, int mode) {
        for (size_t i = 0; i < n; ++i) {
            ArrayPlan &a = plan->arrays[i];
            if (cls(a) == c && !a.ternary() && (a.algo_auto || a.algo == SWDFT_ALGO_TREE_F32)) {
                a.batch_mode = mode;
                a.algo = mode == kBatchSolo ? own_algo[i] : SWDFT_ALGO_TREE_F32;
            }
        }
    };
    // time shape c in its current forms
    auto time_class = [&](int c, float *ms_out) -> swdft_status {
        plan->pipe_uploaded = false;
        swdft_status st = pipe_ready(plan);  // synchronises the device
        if (st != SWDFT_OK) return st;
        fill_batch(plan, d_in, d_out, ws);
        if (cudaMemcpy(plan->desc_dev, plan->desc_host, plan->desc_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return SWDFT_ERR_CUDA;
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return SWDFT_ERR_CUDA;
            if ((st = launch_batch(plan, plan->desc_dev, d_in, d_out, ws, s, c)) != SWDFT_OK) return st;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return SWDFT_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);  // the first run warms up
        }
        *ms_out = best;
        return SWDFT_OK;
    };
    swdft_status st = SWDFT_OK;
    std::vector<char> done(swdft2d_plan_s::kPz, 0);
    for (size_t i = 0; i < n && st == SWDFT_OK; ++i) {
        const ArrayPlan &a0 = plan->arrays[i];
        const int c = cls(a0);
        if (a0.ternary() || done[(size_t)c] || !(a0.algo_auto || a0.algo == SWDFT_ALGO_TREE_F32)) continue;
        done[(size_t)c] = 1;
        std::vector<int> forms = {kBatchPipe, kBatchSolo};
        if (a0.m1 < kBatchFusedM1) forms.push_back(kBatchFused);
        int best = kBatchPipe;
        float best_ms = 1e30f;
        for (int f : forms) {
            set_form(c, f);
            float ms = 0.f;
            if ((st = time_class(c, &ms)) != SWDFT_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = f;
            }
        }
        set_form(c, best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->pipe_uploaded = false;
    destroy_graph(plan->graph);
    return st;
}

}  // namespace

swdft_status swdft2d_autotune(swdft2d_plan_t plan, const void *const *d_in, void *const *d_out,
                              void *d_workspace, void *stream) {
    if (!plan) return SWDFT_ERR_INVALID_ARG;
    swdft_status st = check_buffers(plan, d_in, d_out, d_workspace);
    if (st != SWDFT_OK) return st;
    if ((st = configure(plan)) != SWDFT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool persistent = (plan->flags & SWDFT_FLAG_PERSISTENT) != 0;
    // arrays with a record in the tuning cache for this GPU take it without timing
    const char *cache = std::getenv("SWDFT_TUNE_CACHE");
    char gpu[256] = "unknown";
    std::vector<char> loaded(plan->arrays.size(), 0);
    if (cache) {
        if (!device_name(gpu, sizeof gpu)) return SWDFT_ERR_CUDA;
        load_tuning(plan, cache, gpu, loaded);
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SWDFT_ERR_CUDA;
    for (size_t i = 0; i < plan->arrays.size(); ++i) {
        ArrayPlan &a = plan->arrays[i];
        if (loaded[i]) continue;
        // an array of the same shape, band and form tuned earlier in this call: same choice
        bool copied = false;
        for (size_t j = 0; j < i && !copied; ++j) {
            const ArrayPlan &b = plan->arrays[j];
            if (b.tuned && b.N0 == a.N0 && b.N1 == a.N1 && b.ld == a.ld && b.n0 == a.n0 && b.n1 == a.n1 &&
                b.dtype == a.dtype && b.q_begin == a.q_begin && b.q_end == a.q_end && b.algo_auto == a.algo_auto &&
                (a.algo_auto || b.algo == a.algo)) {
                a.cfg = b.cfg;
                a.algo = b.algo;
                a.tuned = true;
                copied = true;
            }
        }
        if (copied) continue;
        if (a.algo_auto) a.algo = SWDFT_ALGO_TREE_F32;  // the tree is tuned first, then compared
        default_config(a, plan->sm_count, plan->conc);
        if (a.ternary()) continue;  // one launch shape per ternary kernel: nothing to choose
        const TreeConfig dflt = a.cfg;  // the default, fused or not: timed against the winner below
        TreeConfig base = dflt;
        base.fused = false;  // launch shapes are searched on the two-pass form (its row pass fills z)
        std::vector<TreeConfig> cands;
        for (int cb = std::max(0, std::min(a.m0, 3) - 2); cb <= std::min(a.m0, 3); ++cb)
            for (int groups : {1, 2})
                for (int nc : {4, 8, 12, 16}) {
                    if (a.m0 >= 5 && cb < a.m0 - 3) continue;  // these spill registers
                    TreeConfig c = base;
                    c.col_B = cb;
                    c.col_groups = col_tree_clamp_groups(a.m0, cb, groups);
                    c.col_chunk = col_chunk_for(a, nc);
                    cands.push_back(c);
                }
        for (int rb : {std::min(a.m1, 1), std::min(a.m1, 3)}) {
            TreeConfig c = base;
            c.row_B = rb;
            cands.push_back(c);
        }
        // time one pass (stage 1 = row levels, 2 = column levels) of config c, best of 3, in
        // the array's own workspace region (a persistent plan's) or the plan's first slot
        void *slot = persistent ? static_cast<char *>(d_workspace) + plan->z_off[i] : d_workspace;
        auto time_pass = [&](const TreeConfig &c, int stage, float *ms_out) -> bool {
            a.cfg = c;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                if (enqueue_forward(plan, a, d_in[i], d_out[i], slot, a.q_begin, a.q_end, s,
                                    stage) != cudaSuccess)
                    return false;
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) return false;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_min = std::min(ms_min, ms);
            }
            *ms_out = ms_min;
            return true;
        };
        TreeConfig best_c = base;
        float best_col = 1e30f, best_row = 1e30f;
        bool ok = time_pass(base, 1, &best_row);  // fills z for the column candidates
        for (const TreeConfig &c : cands) {
            float ms = 0.f;
            if (ok && c.row_B == base.row_B) {
                ok = time_pass(c, 2, &ms);
                if (ok && ms < best_col) {
                    best_col = ms;
                    best_c.col_B = c.col_B;
                    best_c.col_groups = c.col_groups;
                    best_c.col_chunk = c.col_chunk;
                }
            }
            if (ok && c.row_B != base.row_B) {
                ok = time_pass(c, 1, &ms);
                if (ok && ms < best_row) {
                    best_row = ms;
                    best_c.row_B = c.row_B;
                }
            }
        }
        // fused form: one kernel, timed as a whole against the two passes
        float best = best_row + best_col;
        if (ok && fused_supported(a.m0, a.m1)) {
            for (int nc : {2, 4, 8, 16}) {
                TreeConfig c = best_c;
                c.fused = true;
                c.col_groups = 1;
                c.col_chunk = col_chunk_for(a, nc);
                float ms = 0.f;
                ok = time_pass(c, 2, &ms);
                if (!ok) break;
                if (ms < best) {
                    best = ms;
                    best_c = c;
                }
            }
        }
        // the winner against the default, each timed as a whole forward: the search sums
        // separately timed passes, so it keeps its choice only where the whole is faster too
        if (ok && (best_c.fused != dflt.fused || best_c.col_B != dflt.col_B || best_c.col_groups != dflt.col_groups ||
                   best_c.col_chunk != dflt.col_chunk || best_c.row_B != dflt.row_B || best_c.row_chunk != dflt.row_chunk)) {
            float t_best = 0.f, t_dflt = 0.f;
            ok = time_pass(best_c, 3, &t_best) && time_pass(dflt, 3, &t_dflt);
            if (ok && t_dflt <= t_best) best_c = dflt;
            if (ok) best = std::min(t_best, t_dflt);
        }
        if (!ok) {
            a.cfg = dflt;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return SWDFT_ERR_CUDA;
        }
        a.cfg = best_c;
        a.tuned = true;
        // tree or dense contraction: with SWDFT_ALGO_AUTO, the split-bf16 tensor-core form (the
        // one within the 1e-5 bar) competes with the tuned tree on the whole forward
        if (a.algo_auto && a.tc_eligible()) {
            a.algo = SWDFT_ALGO_TC_BF16X3;
            float ms = 0.f;
            ok = time_pass(best_c, 3, &ms);
            if (!ok || ms >= best) a.algo = SWDFT_ALGO_TREE_F32;
            else best = ms;
            if (!ok) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return SWDFT_ERR_CUDA;
            }
        }
        if (cache) {
            if (FILE *f = std::fopen(cache, "a")) {
                write_tune_record(f, gpu, a, best_c, best);
                std::fclose(f);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    destroy_graph(plan->graph);
    plan->pipe_uploaded = false;  // a persistent plan's tiles follow the tuned chunks
    // a persistent plan then picks, per window shape, the kernels its arrays share or their
    // own (just tuned) launches
    return persistent ? autotune_batch(plan, d_in, d_out, d_workspace, s) : SWDFT_OK;
}

swdft_status swdft2d_inject_alloc_failure(int64_t after) {
    swdft::g_alloc_budget.store(after < 0 ? -1 : after, std::memory_order_relaxed);
    return SWDFT_OK;
}

swdft_status swdft2d_selftest_wait_timeout(int32_t polls, void *stream) {
    if (polls < 1 || polls > 4096) return SWDFT_ERR_INVALID_ARG;
    return launch_wait_timeout_probe((uint32_t)polls, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SWDFT_OK
               : SWDFT_ERR_CUDA;
}

swdft_status swdft2d_load_tuning(swdft2d_plan_t plan, const char *path, const char *gpu_name,
                                 int32_t *applied) {
    if (applied) *applied = 0;
    if (!plan || !path) return SWDFT_ERR_INVALID_ARG;
    char gpu[256];
    if (gpu_name) {
        std::snprintf(gpu, sizeof gpu, "%s", gpu_name);
    } else if (!device_name(gpu, sizeof gpu)) {
        return SWDFT_ERR_CUDA;
    }
    std::vector<char> loaded;
    const int n = load_tuning(plan, path, gpu, loaded);
    if (applied) *applied = n;
    return SWDFT_OK;
}

swdft_status swdft2d_check_device(void) {
    int status = 0, probe = 0, col = 0, pipe = 0;
    if (tc_status(&status, true) != cudaSuccess || probe_status(&probe, true) != cudaSuccess ||
        col_tma_status(&col, true) != cudaSuccess || batch_pipe_status(&pipe, true) != cudaSuccess)
        return SWDFT_ERR_CUDA;
    return (status || probe || col || pipe) ? SWDFT_ERR_DEVICE_TIMEOUT : SWDFT_OK;
}

swdft_status swdft2d_debug_batch_wait(int64_t budget_cycles, int32_t poison) {
    if (budget_cycles < 0 || poison < 0) return SWDFT_ERR_INVALID_ARG;
    g_pipe_budget.store(budget_cycles == 0 ? kPipeBudget : budget_cycles, std::memory_order_relaxed);
    g_pipe_poison.store(poison, std::memory_order_relaxed);
    return SWDFT_OK;
}

swdft_status swdft2d_destroy(swdft2d_plan_t plan) {
    if (!plan) return SWDFT_OK;
    destroy_graph(plan->graph);
    if (plan->desc_uploaded) {
        cudaEventSynchronize(plan->desc_uploaded);
        cudaEventDestroy(plan->desc_uploaded);
    }
    if (plan->desc_host) cudaFreeHost(plan->desc_host);
    for (int k = 0; k < kConc; ++k) {
        if (plan->fside[k]) cudaStreamDestroy(plan->fside[k]);
        if (plan->fjoin_ev[k]) cudaEventDestroy(plan->fjoin_ev[k]);
        if (plan->side[k]) cudaStreamDestroy(plan->side[k]);
        if (plan->join_ev[k]) cudaEventDestroy(plan->join_ev[k]);
    }
    if (plan->fork_ev) cudaEventDestroy(plan->fork_ev);
    if (plan->desc_dev) cudaFree(plan->desc_dev);
    if (plan->desc_graph) cudaFree(plan->desc_graph);
    if (plan->pipe_dev) cudaFree(plan->pipe_dev);
    // host-buffer staging, including what a set-up that ran out of memory left behind
    if (plan->io_in) cudaFree(plan->io_in);
    if (plan->io_ws) cudaFree(plan->io_ws);
    for (int k = 0; k < 2; ++k) {
        if (plan->io_out[k]) cudaFree(plan->io_out[k]);
        if (plan->io_done[k]) cudaEventDestroy(plan->io_done[k]);
        if (plan->io_copied[k]) cudaEventDestroy(plan->io_copied[k]);
    }
    if (plan->io_copy) cudaStreamDestroy(plan->io_copy);
    delete plan;
    return SWDFT_OK;
}

}  // extern "C"
