// Forward transform for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocating routine) at all: plug-ins that
// are handed only their input and output buffers by a host application, code that runs
// after a framework has claimed the device memory for its own pool, or real-time paths where
// an allocation's latency or possible failure is not acceptable.  The planned entry points
// need a caller-supplied workspace (the z rows between the row-level and the column-level
// pass) and a plan object; swdft2d_execute_static_scratch needs neither.  It keeps z in a
// fixed array of device memory that is part of this library (kStaticScratchBytes below, held
// on every GPU that loads the library until the process exits) and works through the output
// in bands of window rows whose z fits in that array.
//
// The first call on a device looks up the array's device address on that device
// (cudaGetSymbolAddress) and its SM count, so make that first call before any stream
// capture.  Both are kept for the life of the process: a cudaDeviceReset (or anything else
// that destroys the device's primary context) unloads the array and leaves the kept address
// dangling, so this entry point must not be called on a device after it was reset.  Every call
// shares the one array: calls that overlap on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.  The array keeps the last call's
// contents; nothing in it needs to start at zero (the row pass writes every z row the column
// pass reads for a stored window).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "swdft2d.h"
#include "swdft_internal.h"

namespace {

// 32 MiB: one band needs (3*n0/2 + rows - 1) * P1 * n1 * 8 bytes of z.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 128;
void *g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_static_scratch on the current device and its SM count, looked up once
// per device.  (In host code the symbol itself is only a host-side stand-in, never a device
// address.)
swdft_status scratch_address(void **out, int *sm_count) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWDFT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SWDFT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return SWDFT_ERR_CUDA;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return SWDFT_ERR_CUDA;
        g_sm_count[dev] = sms;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    *sm_count = g_sm_count[dev];
    return SWDFT_OK;
}

// n = 3^b 2^a with b >= 1: a side plans build a ternary or mixed-radix tree for
bool radix3_family(int64_t n) {
    if (n < 3 || n % 3 != 0) return false;
    while (n % 3 == 0) n /= 3;
    while (n % 2 == 0) n /= 2;
    return n == 1;
}

int log2_pow2(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while ((int64_t(1) << m) < n) ++m;
    return (int64_t(1) << m) == n ? m : -1;
}

}  // namespace

extern "C" swdft_status swdft2d_execute_static_scratch(const void *d_in, int64_t N0, int64_t N1,
                                                       int64_t ld, int32_t n0, int32_t n1,
                                                       int32_t dtype, int32_t norm, void *d_out,
                                                       void *stream) {
    using namespace swdft;
    if (!d_in || !d_out) return SWDFT_ERR_INVALID_ARG;
    if (N0 < 1 || N1 < 1 || n0 < 1 || n1 < 1) return SWDFT_ERR_INVALID_ARG;
    if (dtype != SWDFT_R32 && dtype != SWDFT_C64) return SWDFT_ERR_INVALID_ARG;
    if (norm < SWDFT_NORM_UNITARY || norm > SWDFT_NORM_INV_N) return SWDFT_ERR_INVALID_ARG;
    const int m0 = log2_pow2(n0), m1 = log2_pow2(n1);
    // radix-2 trees only: ternary and mixed-radix windows (which plans accept) are not offered here
    if ((m0 < 0 && radix3_family(n0)) || (m1 < 0 && radix3_family(n1))) return SWDFT_ERR_UNSUPPORTED;
    if (m0 < 0 || m1 < 0) return SWDFT_ERR_NOT_POW2;
    if (n0 > N0 || n1 > N1) return SWDFT_ERR_WINDOW_TOO_LARGE;
    if (m0 > kMaxLog2 || m1 > kMaxLog2) return SWDFT_ERR_UNSUPPORTED;
    if (ld == 0) ld = N1;
    if (ld < N1) return SWDFT_ERR_INVALID_ARG;
    const size_t elem = dtype == SWDFT_C64 ? sizeof(float2) : sizeof(float);
    if ((uintptr_t)d_in % elem != 0 || (uintptr_t)d_out % 16 != 0) return SWDFT_ERR_INVALID_ARG;

    const int64_t P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    const size_t zrow_bytes = (size_t)P1 * (size_t)n1 * sizeof(float2);
    const int64_t z_rows_fit = (int64_t)(kStaticScratchBytes / zrow_bytes);
    const int64_t pad = n0 / 2;
    const int64_t band = z_rows_fit - pad - (n0 - 1);  // window rows per band
    if (band < 1) return SWDFT_ERR_WORKSPACE;           // one band does not fit the array

    void *scratch = nullptr;
    int sm_count = 0;
    swdft_status st = scratch_address(&scratch, &sm_count);
    if (st != SWDFT_OK) return st;

    float2 om64[kMaxN];
    make_omega(kMaxN, om64);
    const double nn = (double)n0 * (double)n1;
    const float scale = norm == SWDFT_NORM_NONE ? 1.0f
                        : norm == SWDFT_NORM_INV_N ? (float)(1.0 / nn) : (float)(1.0 / std::sqrt(nn));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float2 *z = static_cast<float2 *>(scratch) + pad * P1 * n1;
    const size_t out_row = (size_t)P1 * n0 * n1;

    for (int64_t q = 0; q < P0; q += band) {
        const int64_t rows_out = std::min(band, P0 - q);
        RowTreeArgs r;
        r.x = d_in;
        r.ld = ld;
        r.cplx = dtype == SWDFT_C64;
        r.r_base = q;
        r.rows = rows_out + n0 - 1;
        r.P1 = P1;
        r.m1 = m1;
        r.z = z;
        r.om64 = om64;
        // the launch shapes the planned entry points use for a band of this size
        r.B = default_row_B(m1);
        r.chunk = default_row_chunk(P1, r.rows, int64_t(1) << r.B, n1);
        if (launch_row_tree(r, s) != cudaSuccess) return SWDFT_ERR_CUDA;
        ColTreeArgs c;
        c.z = z;
        c.P1 = P1;
        c.rows_out = rows_out;
        c.m0 = m0;
        c.m1 = m1;
        c.out = static_cast<float2 *>(d_out) + (size_t)q * out_row;
        c.scale = scale;
        c.om64 = om64;
        c.B = default_col_B(m0);
        c.chunk = default_col_chunk(rows_out, n0, default_col_nchunks(P1 * n1, sm_count, false));
        c.groups = 1;
        if (launch_col_tree(c, s) != cudaSuccess) return SWDFT_ERR_CUDA;
    }
    return SWDFT_OK;
}
