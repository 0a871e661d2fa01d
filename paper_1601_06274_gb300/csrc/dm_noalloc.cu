// Allocation-free variant of one Dual MM pass (dm_discrete_pass_noalloc).
//
// Who needs it: callers that must not allocate device memory at all -- for
// example a host process whose memory budget is fixed up front, an embedded
// or real-time pipeline that forbids allocation after start-up, or code
// running where cudaMalloc is unavailable or would change a memory pool's
// accounting.  dm_create + dm_bind_workspace needs a caller-allocated
// workspace; this entry point needs none: the caller passes only its inputs
// and outputs, and the pass's scratch (the chain messages, the penalty taps
// and an error word) lives in the fixed file-scope array below.
//
// The array is a static __device__ object: every GPU that loads libdm.so
// holds its kScratchBytes (32 MiB) until the process exits.  In host code the
// symbol is only a host-side stand-in, never a device address, so the device
// address is looked up with cudaGetSymbolAddress once per device (on the first
// call made with that device current) and passed to the kernel.
//
// Every call shares the one array and leaves its contents behind; the kernel
// zeroes what must start at zero (the boundary messages) and rewrites
// everything else before reading it.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
//
// The penalty taps are built on the host and reach the array through the
// parameters of a small kernel (passed by value), so no enqueued operation
// reads host memory.

#include <cstring>
#include <mutex>

#include "dm_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
constexpr size_t kTapsBytes = 256 * dm::kTapW * sizeof(int32_t);  // 8 KiB
constexpr size_t kMsgOffset = kTapsBytes + 256;                  // 256-byte aligned

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// the taps table, passed by value as a kernel parameter (8 KiB)
struct TapsTable {
    int32_t v[256 * dm::kTapW];
};

__global__ void store_taps_kernel(const TapsTable t, int32_t* dst)
{
    for (int i = threadIdx.x; i < 256 * dm::kTapW; i += blockDim.x) dst[i] = t.v[i];
}

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (set up once)
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return DM_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DM_OK;
}

}  // namespace

extern "C" DM_API int dm_discrete_pass_noalloc(int H, int W, int L, const dm_params* p,
                                               int which, const uint8_t* d_cost,
                                               const uint8_t* d_wedge, const int32_t* d_lam_in,
                                               int32_t* d_lam_out, int32_t* d_err, void* stream)
{
    if (p == nullptr || d_lam_in == nullptr || d_lam_out == nullptr || d_wedge == nullptr ||
        d_err == nullptr || d_lam_in == d_lam_out)
        return DM_ERR_ARG;
    if (which != 0 && which != 1) return DM_ERR_ARG;
    if (which == 0 && d_cost == nullptr) return DM_ERR_ARG;
    if (H < 1 || W < 1 || L < 2 || L > 256 || H > 65535 || W > 65535) return DM_ERR_ARG;
    if (!dm::params_valid(*p)) return DM_ERR_ARG;
    const int lpt = L <= 32 ? 1 : (L <= 64 ? 2 : (L <= 128 ? 4 : 8));
    const int KP = 32 * lpt;
    // fmsg and bmsg: one int32 message of KP labels per chain node each
    const size_t msg_bytes = (size_t)H * W * KP * sizeof(int32_t);
    if (kMsgOffset + 2 * msg_bytes > kScratchBytes) return DM_ERR_WORKSPACE;

    // penalty taps for every omega, built on the host
    TapsTable taps;
    int radius = 1;
    long long p2_all = 0;  // the largest cap omega C over every usable omega
    for (int om = 0; om < 256; ++om) {
        int32_t* row = &taps.v[om * dm::kTapW];
        const int r = dm::penalty_taps(om, L, *p, row);
        if (r < 0 && (om == p->w_hi || om == p->w_lo)) return DM_ERR_ARG;
        if (r > radius) radius = r;
        if (row[dm::kTapValid] && row[dm::kTapP2] > p2_all) p2_all = row[dm::kTapP2];
    }
    // the int32 kernel's messages stay below 2^30 when (largest unary + 4 omega C)
    // times the chain length does; with the uint8 costs and lambda_in = 0 this is
    // the bound the context path admits
    const long long n = (H > W ? H : W) + 1;
    if ((255LL + 4 * p2_all) * n >= (1LL << 30)) return DM_ERR_RANGE;

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != DM_OK) return rc;
    unsigned char* s = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t* err = d_err;
    store_taps_kernel<<<1, 256, 0, st>>>(taps, reinterpret_cast<int32_t*>(s));
    if (cudaGetLastError() != cudaSuccess) return DM_ERR_CUDA;

    dm::DmmArgs a{};
    a.which = which;
    a.H = H;
    a.W = W;
    a.L = L;
    a.KP = KP;
    a.cost = d_cost;
    a.lam_in = d_lam_in;
    a.lam_out = d_lam_out;
    a.wedge = d_wedge;
    a.fmsg = reinterpret_cast<int32_t*>(s + kMsgOffset);
    a.bmsg = reinterpret_cast<int32_t*>(s + kMsgOffset + msg_bytes);
    a.taps = reinterpret_cast<const int32_t*>(s);
    a.err = err;
    a.labels = nullptr;
    a.lb = nullptr;
    if (dm::launch_dmm_pass(a, lpt, radius, st) != cudaSuccess) return DM_ERR_CUDA;
    return DM_OK;
}
