// Two-sided consistency check (Sec. 4.1.1 of arXiv 1601.06274: the outliers
// that the truncated regulariser lets through are removed by checking the left
// and the right view against each other; the caption of Table 1 puts the whole
// procedure at twice the one-view time).
//
// The right view's disparity comes from the unchanged path run on the mirrored
// pair (cost.cu, MIRROR): um[y][x'] is the right view's disparity at column
// W-1-x'.  One thread per left pixel (y, x) with d = ul[y][x]: the counterpart
// column is xr = x - rint(d) (nearest, ties to even), and the pixel passes when
// 0 <= xr < W and |d - uR(y, xr)| <= max_diff, evaluated in single precision.
// ok = 1 or 0; out = d or -1; ur (nullable) = the right view's disparity in
// its own columns.  8 B read and 5 B written per pixel (13 B with ur): bound
// by HBM, a few microseconds at 1242x375.

#include "dm_internal.cuh"

namespace dm {
namespace {

__global__ void lr_check_kernel(const float* __restrict__ ul, const float* __restrict__ um, int H,
                                int W, float max_diff, uint8_t* __restrict__ ok,
                                float* __restrict__ out, float* __restrict__ ur)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)H * W) return;
    const int y = (int)(i / W);
    const int x = (int)(i - (long long)y * W);
    const float* row = um + (long long)y * W;
    const float d = ul[i];
    bool pass = false;
    if (isfinite(d) && fabsf(d) < 1.0e9f) {
        const long long xr = (long long)x - (long long)rintf(d);
        if (xr >= 0 && xr < W) pass = fabsf(d - row[W - 1 - xr]) <= max_diff;
    }
    ok[i] = pass ? 1 : 0;
    out[i] = pass ? d : -1.0f;
    if (ur != nullptr) ur[i] = row[W - 1 - x];
}

}  // namespace

cudaError_t launch_lr_check(const float* ul, const float* um, int H, int W, float max_diff,
                            uint8_t* ok, float* out, float* ur, cudaStream_t s)
{
    const long long n = (long long)H * W;
    const int threads = 256;
    const long long blocks = (n + threads - 1) / threads;
    lr_check_kernel<<<(unsigned)blocks, threads, 0, s>>>(ul, um, H, W, max_diff, ok, out, ur);
    return cudaGetLastError();
}

}  // namespace dm
