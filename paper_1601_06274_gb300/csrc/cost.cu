// Census transform, edge weights and matching-cost volume (Sec. 3.1 of
// arXiv 1601.06274: census on a small patch, pixel-wise Hamming distance;
// Sec. 1: the cost is precomputed for every label).
//
// census: one thread per pixel, both images in one launch (blockIdx.z picks
//   the image); the 5x5 (or 3x3) window is read through L1 with
//   clamp-to-edge indices.  Bit k is the k-th neighbour in raster order,
//   centre skipped, set when I(neighbour) < I(centre).  The left image's
//   threads also write the edge weights omega (Sec. 2.1: image dependent,
//   weaker across intensity edges).  MIRROR computes the same for the mirrored
//   pair (the right image, columns reversed, as the reference; the left image,
//   columns reversed, as the other view): the right view's problem of the
//   two-sided check (Sec. 4.1.1), with no extra pass over the images.
// cost:   c[y][x][l] = popcount(cL[y][x] ^ cR[y][x-l]) or win*win-1 when
//   x - l < 0.  One thread writes 16 consecutive labels of one pixel as a
//   single 16-byte store, so a warp writes 512 contiguous bytes.

#include "dm_internal.cuh"

namespace dm {
namespace {

template <int WIN, bool MIRROR>
__global__ void census_edges_kernel(const uint8_t* __restrict__ left,
                                    const uint8_t* __restrict__ right, int H, int W, int T,
                                    int w_hi, int w_lo, uint32_t* __restrict__ census,
                                    uint8_t* __restrict__ wh, uint8_t* __restrict__ wv)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int img = blockIdx.z;
    if (x >= W || y >= H) return;
    // column xx of the (possibly mirrored) image: I[row + col(xx)]
    const uint8_t* I = (img == 0) != MIRROR ? left : right;
    auto col = [W](int xx) { return MIRROR ? W - 1 - xx : xx; };
    constexpr int r = WIN / 2;
    const int centre = I[y * W + col(x)];
    uint32_t code = 0;
    int bit = 0;
#pragma unroll
    for (int dy = -r; dy <= r; ++dy) {
        const int yy = min(max(y + dy, 0), H - 1);
#pragma unroll
        for (int dx = -r; dx <= r; ++dx) {
            if (dy == 0 && dx == 0) continue;
            const int xx = min(max(x + dx, 0), W - 1);
            code |= (uint32_t)(I[yy * W + col(xx)] < centre) << bit;
            ++bit;
        }
    }
    census[(size_t)img * H * W + (size_t)y * W + x] = code;
    if (img == 0) {
        const size_t i = (size_t)y * W + x;
        uint8_t a = 0, b = 0;
        if (x + 1 < W) a = (uint8_t)(abs(centre - (int)I[y * W + col(x + 1)]) < T ? w_hi : w_lo);
        if (y + 1 < H) b = (uint8_t)(abs(centre - (int)I[(y + 1) * W + col(x)]) < T ? w_hi : w_lo);
        wh[i] = a;
        wv[i] = b;
    }
}

template <typename CT>
__global__ void cost_kernel(const uint32_t* __restrict__ cl, const uint32_t* __restrict__ cr,
                            int H, int W, int L, int maxc, CT* __restrict__ cost)
{
    // one thread: pixel p, labels [16 g, 16 g + 16)
    const int groups = (L + 15) >> 4;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)H * W * groups;
    if (t >= total) return;
    const int g = (int)(t % groups);
    const long long p = t / groups;
    const int x = (int)(p % W);
    const uint32_t a = cl[p];
    const int l0 = g << 4;
    uint32_t v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int l = l0 + k;
        const int xr = x - l;
        v[k] = xr >= 0 ? (uint32_t)__popc(a ^ cr[p - l]) : (uint32_t)maxc;
    }
    CT* dst = cost + p * L + l0;
    if ((L & 15) == 0) {
        if constexpr (sizeof(CT) == 1) {
            uint4 w;
            w.x = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
            w.y = v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24);
            w.z = v[8] | (v[9] << 8) | (v[10] << 16) | (v[11] << 24);
            w.w = v[12] | (v[13] << 8) | (v[14] << 16) | (v[15] << 24);
            *reinterpret_cast<uint4*>(dst) = w;
        } else {
            uint4 w0, w1;
            w0.x = v[0] | (v[1] << 16);
            w0.y = v[2] | (v[3] << 16);
            w0.z = v[4] | (v[5] << 16);
            w0.w = v[6] | (v[7] << 16);
            w1.x = v[8] | (v[9] << 16);
            w1.y = v[10] | (v[11] << 16);
            w1.z = v[12] | (v[13] << 16);
            w1.w = v[14] | (v[15] << 16);
            reinterpret_cast<uint4*>(dst)[0] = w0;
            reinterpret_cast<uint4*>(dst)[1] = w1;
        }
    } else {
        for (int k = 0; k < 16 && l0 + k < L; ++k) dst[k] = (CT)v[k];
    }
}

}  // namespace

cudaError_t launch_census_edges(const uint8_t* left, const uint8_t* right, int H, int W, int win,
                                int T, int w_hi, int w_lo, uint32_t* census, uint8_t* wh,
                                uint8_t* wv, bool mirror, cudaStream_t s)
{
    dim3 blk(32, 8);
    dim3 grd((W + 31) / 32, (H + 7) / 8, 2);
    auto k = win == 5 ? (mirror ? census_edges_kernel<5, true> : census_edges_kernel<5, false>)
                      : (mirror ? census_edges_kernel<3, true> : census_edges_kernel<3, false>);
    k<<<grd, blk, 0, s>>>(left, right, H, W, T, w_hi, w_lo, census, wh, wv);
    return cudaGetLastError();
}

cudaError_t launch_cost(const uint32_t* census, int H, int W, int L, int maxc, void* cost,
                        int cost_bytes, cudaStream_t s)
{
    const long long total = (long long)H * W * ((L + 15) / 16);
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    if (cost_bytes == 2)
        cost_kernel<uint16_t><<<(unsigned)blocks, threads, 0, s>>>(
            census, census + (size_t)H * W, H, W, L, maxc, static_cast<uint16_t*>(cost));
    else
        cost_kernel<uint8_t><<<(unsigned)blocks, threads, 0, s>>>(
            census, census + (size_t)H * W, H, W, L, maxc, static_cast<uint8_t*>(cost));
    return cudaGetLastError();
}

}  // namespace dm
