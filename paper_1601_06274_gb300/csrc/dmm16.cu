// Dual MM pass with packed 16-bit arithmetic: dispatch over the label classes
// of the lane-group kernel (dmg_g*_*.cu from dmg_impl.cuh) and of the
// one-warp-per-chain kernel (dmm16_np*_*.cu from dmm16_impl.cuh), and the
// conversion kernels between the packed dual storage and int32.

#include <climits>

#include "dm_internal.cuh"

namespace dm {

template <int NP, typename DT>
cudaError_t launch16(const Dmm16Args& a, int radius, cudaStream_t s);
template <int NP, typename DT>
cudaError_t launch16_batch(const Batch16Args& b, int radius, bool pad, cudaStream_t s);
template <int G, typename DT>
cudaError_t launch_g(const Dmm16Args& a, int radius, cudaStream_t s);
template <int G, typename DT>
cudaError_t launch_g_batch(const Batch16Args& b, int radius, cudaStream_t s);

namespace {

__global__ void validate_edges_kernel(const uint8_t* __restrict__ wh, const uint8_t* __restrict__ wv,
                                      int H, int W, const int32_t* __restrict__ taps,
                                      int32_t* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * W) return;
    const int x = i % W, y = i / W;
    bool bad = false;
    if (x + 1 < W) bad |= taps[(int)wh[i] * kTapW + kTapValid] == 0;
    if (y + 1 < H) bad |= taps[(int)wv[i] * kTapW + kTapValid] == 0;
    if (bad) atomicOr(err, kDevErrBadOmega);
}

__device__ __forceinline__ int cost_at(const void* cost, int cost_bytes, long long t)
{
    return cost_bytes == 2 ? (int)static_cast<const uint16_t*>(cost)[t]
                           : (int)static_cast<const uint8_t*>(cost)[t];
}

// out = base + delta - (cost if given): lambda_h, or lambda_v from c + lambda_v
__global__ void duals_to_i32_kernel(const int32_t* __restrict__ base, const void* __restrict__ delta,
                                    int delta_bytes, const void* __restrict__ cost, int cost_bytes,
                                    long long n_px, int L, int32_t* __restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_px * L) return;
    const long long px = t / L;
    const int d = delta_bytes == 1 ? (int)static_cast<const uint8_t*>(delta)[t]
                                   : (int)static_cast<const int16_t*>(delta)[t];
    out[t] = base[px] + d - (cost != nullptr ? cost_at(cost, cost_bytes, t) : 0);
}

// cold start of the 16-bit path: the horizontal unary c + lambda_v with lambda_v = 0
__global__ void theta_h_init_kernel(const void* __restrict__ cost, int cost_bytes,
                                    int32_t* __restrict__ base, void* __restrict__ delta,
                                    int delta_bytes, long long n_px, int L)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_px) base[t] = 0;
    if (t >= n_px * L) return;
    const int c = cost_at(cost, cost_bytes, t);
    if (delta_bytes == 1) static_cast<uint8_t*>(delta)[t] = (uint8_t)c;
    else static_cast<int16_t*>(delta)[t] = (int16_t)c;
}

// warm start of the 16-bit path: the horizontal unary c + lambda_v for a new
// cost volume c and int32 lambda_v, one warp per pixel: base = the minimum over
// the labels rounded down to even (the kernel's halving commutes only with
// even shifts), deltas above it; a span the deltas cannot hold sets
// kDevErrRange
__global__ void theta_h_from_i32_kernel(const int32_t* __restrict__ lam_v,
                                        const void* __restrict__ cost, int cost_bytes,
                                        int32_t* __restrict__ base, void* __restrict__ delta,
                                        int delta_bytes, long long n_px, int L,
                                        int32_t* __restrict__ err)
{
    const long long px = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (px >= n_px) return;
    const long long row = px * L;
    int mn = INT_MAX, mx = INT_MIN;
    for (int l = lane; l < L; l += 32) {
        const int v = lam_v[row + l] + cost_at(cost, cost_bytes, row + l);
        mn = min(mn, v);
        mx = max(mx, v);
    }
    mn = __reduce_min_sync(0xffffffffu, mn) & ~1;
    mx = __reduce_max_sync(0xffffffffu, mx);
    const int cap = delta_bytes == 1 ? 255 : 16000;
    if (mx - mn > cap) {
        if (lane == 0) atomicOr(err, kDevErrRange);
        return;
    }
    for (int l = lane; l < L; l += 32) {
        const int d = lam_v[row + l] + cost_at(cost, cost_bytes, row + l) - mn;
        if (delta_bytes == 1) static_cast<uint8_t*>(delta)[row + l] = (uint8_t)d;
        else static_cast<int16_t*>(delta)[row + l] = (int16_t)d;
    }
    if (lane == 0) base[px] = mn;
}

}  // namespace

cudaError_t launch_dmm16_pass(const Dmm16Args& a, int np, int radius, int delta_bytes,
                              cudaStream_t s)
{
    if (delta_bytes == 1) {
        if (np == 1) return launch16<1, uint8_t>(a, radius, s);
        if (np == 2) return launch16<2, uint8_t>(a, radius, s);
        return launch16<4, uint8_t>(a, radius, s);
    }
    if (np == 1) return launch16<1, int16_t>(a, radius, s);
    if (np == 2) return launch16<2, int16_t>(a, radius, s);
    return launch16<4, int16_t>(a, radius, s);
}

cudaError_t launch_dmg_pass(const Dmm16Args& a, int g, int radius, int delta_bytes, cudaStream_t s)
{
    if (delta_bytes == 1) {
        switch (g) {
            case 1: return launch_g<1, uint8_t>(a, radius, s);
            case 2: return launch_g<2, uint8_t>(a, radius, s);
            case 4: return launch_g<4, uint8_t>(a, radius, s);
            case 8: return launch_g<8, uint8_t>(a, radius, s);
            default: return launch_g<16, uint8_t>(a, radius, s);
        }
    }
    switch (g) {
        case 1: return launch_g<1, int16_t>(a, radius, s);
        case 2: return launch_g<2, int16_t>(a, radius, s);
        case 4: return launch_g<4, int16_t>(a, radius, s);
        case 8: return launch_g<8, int16_t>(a, radius, s);
        default: return launch_g<16, int16_t>(a, radius, s);
    }
}

// kernels one lane-group pass launches: 2 when launch_g splits it (a pool is
// given, from 128 labels on except the 128-label vertical pass, and the chains
// reach level KL + 1 with segments of 5 or more nodes; KL = log2 of the groups
// of an 8-warp CTA), else 1
int dmg_pass_kernels(const Dmm16Args& a, int g)
{
    if (a.pool == nullptr || g < 8 || (g == 8 && a.which == 1)) return 1;
    const int kl = g == 8 ? 5 : 4;
    const int n = a.which == 0 ? a.W : a.H;
    return n > 4 && ((n + (1 << kl) - 1) >> kl) >= 5 ? 2 : 1;
}

cudaError_t launch_dmg_batch(const Batch16Args& b, int g, int radius, int delta_bytes, cudaStream_t s)
{
    if (delta_bytes == 1) {
        switch (g) {
            case 1: return launch_g_batch<1, uint8_t>(b, radius, s);
            case 2: return launch_g_batch<2, uint8_t>(b, radius, s);
            case 4: return launch_g_batch<4, uint8_t>(b, radius, s);
            case 8: return launch_g_batch<8, uint8_t>(b, radius, s);
            default: return launch_g_batch<16, uint8_t>(b, radius, s);
        }
    }
    switch (g) {
        case 1: return launch_g_batch<1, int16_t>(b, radius, s);
        case 2: return launch_g_batch<2, int16_t>(b, radius, s);
        case 4: return launch_g_batch<4, int16_t>(b, radius, s);
        case 8: return launch_g_batch<8, int16_t>(b, radius, s);
        default: return launch_g_batch<16, int16_t>(b, radius, s);
    }
}

cudaError_t launch_dmm16_batch(const Batch16Args& b, int np, int radius, bool pad, int delta_bytes,
                               cudaStream_t s)
{
    if (delta_bytes == 1) {
        if (np == 1) return launch16_batch<1, uint8_t>(b, radius, pad, s);
        if (np == 2) return launch16_batch<2, uint8_t>(b, radius, pad, s);
        return launch16_batch<4, uint8_t>(b, radius, pad, s);
    }
    if (np == 1) return launch16_batch<1, int16_t>(b, radius, pad, s);
    if (np == 2) return launch16_batch<2, int16_t>(b, radius, pad, s);
    return launch16_batch<4, int16_t>(b, radius, pad, s);
}

cudaError_t launch_validate_edges(const uint8_t* wh, const uint8_t* wv, int H, int W,
                                  const int32_t* taps, int32_t* err, cudaStream_t s)
{
    const int n = H * W;
    validate_edges_kernel<<<(n + 255) / 256, 256, 0, s>>>(wh, wv, H, W, taps, err);
    return cudaGetLastError();
}

cudaError_t launch_duals_to_i32(const int32_t* base, const void* delta, int delta_bytes,
                                const void* cost, int cost_bytes, long long n_px, int L,
                                int32_t* out, cudaStream_t s)
{
    const long long total = n_px * L;
    duals_to_i32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        base, delta, delta_bytes, cost, cost_bytes, n_px, L, out);
    return cudaGetLastError();
}

cudaError_t launch_theta_h_init(const void* cost, int cost_bytes, int32_t* base, void* delta,
                                int delta_bytes, long long n_px, int L, cudaStream_t s)
{
    const long long total = n_px * L;
    if (cost_bytes == 1 && delta_bytes == 1) {
        // the deltas are the cost bytes themselves, over a zero base
        cudaError_t e = cudaMemsetAsync(base, 0, (size_t)n_px * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(delta, cost, (size_t)total, cudaMemcpyDeviceToDevice, s);
    }
    theta_h_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        cost, cost_bytes, base, delta, delta_bytes, n_px, L);
    return cudaGetLastError();
}

cudaError_t launch_theta_h_from_i32(const int32_t* lam_v, const void* cost, int cost_bytes,
                                    int32_t* base, void* delta, int delta_bytes, long long n_px,
                                    int L, int32_t* err, cudaStream_t s)
{
    const long long threads = n_px * 32;
    theta_h_from_i32_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        lam_v, cost, cost_bytes, base, delta, delta_bytes, n_px, L, err);
    return cudaGetLastError();
}

}  // namespace dm
