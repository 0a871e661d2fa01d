// Continuous refinement of arXiv 1601.06274 (Sec. 2.4 and 3.1): Valkonen's
// non-linear primal-dual iterates (Eq. cont_iterates) for
//   min_{u,q} max_p <Au, p - q> - R+*(p) + R-*(q) + D~(u),
// with the difference-of-convex split r = r_{eps,delta} - r_{0,C+delta-eps delta}
// (Eq. r-decompose), the convexified data term D~ of Sec. 3.1 and the warping
// loop that re-linearises D around the current u.
//
// Layout: all state is float32 [H][W].  An edge e = (i, j) with j the right
// (or lower) neighbour is stored at pixel i in *_h (or *_v); (Au)_e = u_i - u_j.
//
// One iteration is one kernel (Jacobi in the pixels, ping-pong buffers): a
// 32x8 tile first computes u+ = prox_{tau D~}(u - tau A^T (p - q)) on the tile
// and a one-pixel halo to the right and below (from the old p, q), then the
// edges of the tile:
//   q+ = prox_{tau R-*}(q + tau A u),  p+ = prox_{sigma R+*}(p + sigma A (2u+ - u)).
// The cost samples are uint8 (census) or float32 (a caller's cost volume), the
// data weight a scalar or a per-pixel map.

#include "dm_internal.cuh"

namespace dm {
namespace {

constexpr int kTX = 32, kTY = 8;

__device__ __forceinline__ float cost_at(const PdArgs& A, size_t i)
{
    return A.costf != nullptr ? __ldg(A.costf + i) : (float)__ldg(A.cost + i);
}

// D_i(x): linear interpolation of the cost samples of pixel px with the argument
// clamped to [0, L-1]
__device__ __forceinline__ float interp(const PdArgs& A, size_t px, float x)
{
    const int L = A.L;
    x = fminf(fmaxf(x, 0.0f), (float)(L - 1));
    int k = (int)floorf(x);
    if (k > L - 2) k = L - 2;
    if (k < 0) k = 0;
    const float t = x - (float)k;
    const float c0 = cost_at(A, px * L + k);
    const float c1 = cost_at(A, px * L + k + 1);
    return c0 + t * (c1 - c0);
}

__device__ __forceinline__ float alpha_at(const PdArgs& A, int i)
{
    return A.alpha_px != nullptr ? __ldg(A.alpha_px + i) : A.alpha;
}

__global__ void init_u_kernel(const uint16_t* __restrict__ labels, float* __restrict__ u, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = (float)labels[i];
}

__global__ void zero_kernel(float* __restrict__ p, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.0f;
}

// Linearisation of the data term around u0 = u (Sec. 3.1): slopes s1 (left of
// u0) and s2 (right of u0), both set to their mean when s2 < s1, and the box
// [u0 - h, u0 + h] intersected with [0, L-1].
__global__ void linearise_kernel(const PdArgs A)
{
    const int n = A.H * A.W;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float u0 = A.u[i];
    const float d0 = interp(A, i, u0);
    const float dm = interp(A, i, u0 - A.h);
    const float dp = interp(A, i, u0 + A.h);
    const float al = alpha_at(A, i);
    float s1 = al * (d0 - dm) / A.h;
    float s2 = al * (dp - d0) / A.h;
    if (s2 < s1) {
        s1 = 0.5f * (s1 + s2);
        s2 = s1;
    }
    A.u0[i] = u0;
    A.s1[i] = s1;
    A.s2[i] = s2;
    A.lo[i] = fmaxf(u0 - A.h, 0.0f);
    A.hi[i] = fminf(u0 + A.h, (float)(A.L - 1));
}

// prox of step * (omega r_{a,b})*: identity on |t| <= a omega, else shrink by
// b * step but not below a omega; then clamp to [-omega, omega] (Eq. pprox)
__device__ __forceinline__ float prox_conj(float t, float omega, float a, float b, float step)
{
    const float at = fabsf(t);
    float v = t;
    if (at > a * omega) v = copysignf(fmaxf(a * omega, at - b * step), t);
    return fminf(fmaxf(v, -omega), omega);
}

// u+ at pixel (x, y) from the old state
__device__ __forceinline__ float u_step(const PdArgs& A, int x, int y)
{
    const int W = A.W;
    const int i = y * W + x;
    float div = 0.0f;  // (A^T (p - q))_i
    if (x + 1 < W) div += A.ph[i] - A.qh[i];
    if (x > 0) div -= A.ph[i - 1] - A.qh[i - 1];
    if (y + 1 < A.H) div += A.pv[i] - A.qv[i];
    if (y > 0) div -= A.pv[i - W] - A.qv[i - W];
    const float uh = A.u[i] - A.tau * div;
    const float u0 = A.u0[i];
    const float ts1 = A.tau * A.s1[i];
    const float ts2 = A.tau * A.s2[i];
    float v;
    if (uh > u0 + ts2) v = uh - ts2;
    else if (uh < u0 + ts1) v = uh - ts1;
    else v = u0;
    return fminf(fmaxf(v, A.lo[i]), A.hi[i]);
}

__global__ void __launch_bounds__(kTX * kTY) pd_fused_kernel(const PdArgs A)
{
    __shared__ float s_un[kTY + 1][kTX + 1];  // u+ on the tile and its right/lower halo
    __shared__ float s_u[kTY + 1][kTX + 1];   // old u there
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int W = A.W, H = A.H;
    for (int t = threadIdx.x; t < (kTX + 1) * (kTY + 1); t += kTX * kTY) {
        const int lx = t % (kTX + 1), ly = t / (kTX + 1);
        const int x = x0 + lx, y = y0 + ly;
        if (x < W && y < H) {
            s_un[ly][lx] = u_step(A, x, y);
            s_u[ly][lx] = A.u[y * W + x];
        }
    }
    __syncthreads();
    const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) return;
    const int i = y * W + x;
    const float ui = s_u[ly][lx];
    const float uni = s_un[ly][lx];
    A.u_new[i] = uni;
    const float ei = 2.0f * uni - ui;
    if (x + 1 < W) {
        const float om = A.lambda_r * (float)A.wh[i];
        const float uj = s_u[ly][lx + 1];
        const float ej = 2.0f * s_un[ly][lx + 1] - uj;
        A.qh2[i] = prox_conj(A.qh[i] + A.tau * (ui - uj), om, 0.0f, A.bq, A.tau);
        A.ph2[i] = prox_conj(A.ph[i] + A.sigma * (ei - ej), om, A.ap, A.bp, A.sigma);
    }
    if (y + 1 < H) {
        const float om = A.lambda_r * (float)A.wv[i];
        const float uj = s_u[ly + 1][lx];
        const float ej = 2.0f * s_un[ly + 1][lx] - uj;
        A.qv2[i] = prox_conj(A.qv[i] + A.tau * (ui - uj), om, 0.0f, A.bq, A.tau);
        A.pv2[i] = prox_conj(A.pv[i] + A.sigma * (ei - ej), om, A.ap, A.bp, A.sigma);
    }
}

__device__ __forceinline__ double r_dc(double t, double eps, double delta, double C)
{
    const double at = fabs(t);
    const double rp = at <= delta ? eps * at : at - delta * (1.0 - eps);
    const double bq = C + delta - eps * delta;
    const double rm = at <= bq ? 0.0 : at - bq;
    return rp - rm;
}

constexpr int kEnergyThreads = 256;

// per-block partial sums of E(u) in double, reduced in a fixed order
__global__ void energy_kernel(const PdArgs A, double eps, double delta, double C,
                              double* __restrict__ partial)
{
    __shared__ double sh[kEnergyThreads];
    const int n = A.H * A.W;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = i % A.W, y = i / A.W;
        const float* u = A.u;
        acc += (double)alpha_at(A, i) * (double)interp(A, i, u[i]);
        if (x + 1 < A.W)
            acc += (double)A.lambda_r * A.wh[i] * r_dc((double)u[i] - (double)u[i + 1], eps, delta, C);
        if (y + 1 < A.H)
            acc += (double)A.lambda_r * A.wv[i] * r_dc((double)u[i] - (double)u[i + A.W], eps, delta, C);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kEnergyThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

}  // namespace

int energy_blocks(int H, int W)
{
    const int n = H * W;
    int b = (n + kEnergyThreads - 1) / kEnergyThreads;
    return b > 1024 ? 1024 : b;
}

cudaError_t launch_init_u_from_labels(const uint16_t* labels, float* u, int n, cudaStream_t s)
{
    init_u_kernel<<<(n + 255) / 256, 256, 0, s>>>(labels, u, n);
    return cudaGetLastError();
}

cudaError_t launch_zero_f32(float* p, size_t n, cudaStream_t s)
{
    zero_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_linearise(const PdArgs& a, cudaStream_t s)
{
    const int n = a.H * a.W;
    linearise_kernel<<<(n + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pd_iter(const PdArgs& a, cudaStream_t s)
{
    dim3 grd((a.W + kTX - 1) / kTX, (a.H + kTY - 1) / kTY);
    pd_fused_kernel<<<grd, kTX * kTY, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_energy(const PdArgs& a, double eps, double delta, double C, double* partial,
                          int nblocks, cudaStream_t s)
{
    energy_kernel<<<nblocks, kEnergyThreads, 0, s>>>(a, eps, delta, C, partial);
    return cudaGetLastError();
}

}  // namespace dm
