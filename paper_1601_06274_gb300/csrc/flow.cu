// Optical flow (Sec. 2.2 "Flow" and the appendix section on optical flow of
// arXiv 1601.06274): decoupled discrete layers and the two-component
// refinement with the quadratic data model.
//
// Displacement of pixel (y, x): (d1, d2) = (lo1 + label1, lo2 + label2), d1
// horizontal.  Data cost D(d1, d2) = popcount(census1(y, x) ^ census2(y + d2,
// x + d1)), maxc where the displaced pixel leaves the image.
//
// flow_cost_kernel: the decoupled costs (Eq. flow decoupled costs) p1(l1) =
//   min_l2 D, p2(l2) = min_l1 D, uint8, one warp per pixel: lanes over l1, a
//   loop over l2 whose row minimum is one redux.  The census row of image 2
//   is read coalesced and shared by neighbouring pixels through L1/L2.
// flow_lin_kernel: at the start of each warp, the quadratic model of alpha D
//   at u0 (3x3 samples of the bilinear data term, computed from the census
//   codes: central first and second differences with step h, the mixed term
//   from the four corners, the positive-semidefinite part of Q) and the box
//   [u0 - h, u0 + h] clipped to the label range.
// flow_primal_kernel: u+ = clamp((I + tau Q)^-1 (u^ + tau (Q u0 - L))), u^ =
//   u - tau A^T (p - q) per component (the prox of the quadratic model; the
//   printed formula's denominator is re-derived as the 2x2 solve).
// flow_dual_kernel: per component and edge, q+ = prox_{tau R-*}(q + tau A u),
//   p+ = prox_{sigma R+*}(p + sigma A (2u+ - u)), in place (every edge is owned
//   by one thread and reads only u and u+).
// All refinement state lives in a caller scratch of 23 float arrays.

#include "dm_internal.cuh"

namespace dm {
namespace {

// ---------------------------------------------------------------------------
// decoupled costs
// ---------------------------------------------------------------------------

constexpr int kFlowWarps = 8;

__global__ void __launch_bounds__(kFlowWarps * 32)
flow_cost_kernel(const uint32_t* __restrict__ c1, const uint32_t* __restrict__ c2, int H, int W,
                 int lo1, int K1, int lo2, int K2, int maxc, uint8_t* __restrict__ p1,
                 uint8_t* __restrict__ p2)
{
    __shared__ uint8_t s_p2[kFlowWarps][256];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long px = (long long)blockIdx.x * kFlowWarps + warp;
    if (px >= (long long)H * W) return;
    const int y = (int)(px / W);
    const int x = (int)(px - (long long)y * W);
    const uint32_t a = c1[px];
    const int nj = (K1 + 31) >> 5;  // label groups of 32 per lane (K1 <= 256)
    int m1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) m1[j] = maxc;
    for (int l2 = 0; l2 < K2; ++l2) {
        const int yy = y + lo2 + l2;
        int rowmin = maxc;
        if (yy >= 0 && yy < H) {
            const uint32_t* row = c2 + (long long)yy * W;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j < nj) {
                    const int l1 = lane + 32 * j;
                    const int xx = x + lo1 + l1;
                    int d = maxc;
                    if (l1 < K1 && xx >= 0 && xx < W) d = __popc(a ^ __ldg(row + xx));
                    if (l1 < K1) {
                        m1[j] = min(m1[j], d);
                        rowmin = min(rowmin, d);
                    }
                }
            }
            rowmin = __reduce_min_sync(0xffffffffu, rowmin);
        }
        if (lane == 0) s_p2[warp][l2] = (uint8_t)rowmin;
    }
    __syncwarp();
    uint8_t* o1 = p1 + px * K1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int l1 = lane + 32 * j;
        if (j < nj && l1 < K1) o1[l1] = (uint8_t)m1[j];
    }
    uint8_t* o2 = p2 + px * K2;
    for (int l2 = lane; l2 < K2; l2 += 32) o2[l2] = s_p2[warp][l2];
}

// ---------------------------------------------------------------------------
// refinement
// ---------------------------------------------------------------------------

__device__ __forceinline__ int flow_cost(const FlowArgs& A, int y, int x, int l1, int l2)
{
    const int yy = y + A.lo2 + l2, xx = x + A.lo1 + l1;
    if (yy < 0 || yy >= A.H || xx < 0 || xx >= A.W) return A.maxc;
    return __popc(__ldg(A.c1 + (long long)y * A.W + x) ^ __ldg(A.c2 + (long long)yy * A.W + xx));
}

// bilinear data term at label coordinates (v1, v2), arguments clamped to the ranges
__device__ __forceinline__ float flow_D(const FlowArgs& A, int y, int x, float v1, float v2)
{
    v1 = fminf(fmaxf(v1, 0.0f), (float)(A.K1 - 1));
    v2 = fminf(fmaxf(v2, 0.0f), (float)(A.K2 - 1));
    const int a = min((int)floorf(v1), A.K1 - 2);
    const int b = min((int)floorf(v2), A.K2 - 2);
    const float t = v1 - (float)a, s = v2 - (float)b;
    const float d00 = (float)flow_cost(A, y, x, a, b);
    const float d10 = (float)flow_cost(A, y, x, a + 1, b);
    const float d01 = (float)flow_cost(A, y, x, a, b + 1);
    const float d11 = (float)flow_cost(A, y, x, a + 1, b + 1);
    return (1.0f - t) * (1.0f - s) * d00 + t * (1.0f - s) * d10 + (1.0f - t) * s * d01 +
           t * s * d11;
}

__device__ __forceinline__ float prox_conj_f(float t, float omega, float a, float b, float step)
{
    const float at = fabsf(t);
    const float ao = __fmul_rn(a, omega);
    float v = t;
    if (at > ao) v = copysignf(fmaxf(ao, __fmaf_rn(-b, step, at)), t);
    return fminf(fmaxf(v, -omega), omega);
}

__global__ void flow_init_kernel(FlowArgs A, const uint16_t* __restrict__ lab1,
                                 const uint16_t* __restrict__ lab2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)A.H * A.W) return;
    A.u1[i] = (float)lab1[i];
    A.u2[i] = (float)lab2[i];
    A.ph1[i] = A.pv1[i] = A.qh1[i] = A.qv1[i] = 0.0f;
    A.ph2[i] = A.pv2[i] = A.qh2[i] = A.qv2[i] = 0.0f;
}

__global__ void flow_lin_kernel(FlowArgs A)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)A.H * A.W) return;
    const int y = (int)(i / A.W), x = (int)(i - (long long)y * A.W);
    const float u1 = A.u1[i], u2 = A.u2[i], h = A.h;
    float S[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            S[j][k] = A.alpha * flow_D(A, y, x, u1 + (float)(k - 1) * h, u2 + (float)(j - 1) * h);
    const float L1 = (S[1][2] - S[1][0]) / (2.0f * h);
    const float L2 = (S[2][1] - S[0][1]) / (2.0f * h);
    float q11 = (S[1][2] - 2.0f * S[1][1] + S[1][0]) / (h * h);
    float q12 = (S[2][2] - S[0][2] - S[2][0] + S[0][0]) / (4.0f * h * h);
    float q22 = (S[2][1] - 2.0f * S[1][1] + S[0][1]) / (h * h);
    // positive-semidefinite part: eigenvalues below zero set to zero
    const float m = 0.5f * (q11 + q22);
    const float r = sqrtf(0.25f * (q11 - q22) * (q11 - q22) + q12 * q12);
    const float lp = m + r, lm = m - r;
    if (lm < 0.0f) {
        if (lp <= 0.0f) {
            q11 = q12 = q22 = 0.0f;
        } else {
            float v1, v2;
            if (fabsf(q12) > 0.0f) {
                v1 = q12;
                v2 = lp - q11;
                if (fabsf(v1) + fabsf(v2) == 0.0f) {
                    v1 = lp - q22;
                    v2 = q12;
                }
            } else if (q11 >= q22) {
                v1 = 1.0f;
                v2 = 0.0f;
            } else {
                v1 = 0.0f;
                v2 = 1.0f;
            }
            const float n = sqrtf(v1 * v1 + v2 * v2);
            v1 /= n;
            v2 /= n;
            q11 = lp * v1 * v1;
            q12 = lp * v1 * v2;
            q22 = lp * v2 * v2;
        }
    }
    A.u01[i] = u1;
    A.u02[i] = u2;
    A.L1[i] = L1;
    A.L2[i] = L2;
    A.q11[i] = q11;
    A.q12[i] = q12;
    A.q22[i] = q22;
    A.b1lo[i] = fmaxf(u1 - h, 0.0f);
    A.b1hi[i] = fminf(u1 + h, (float)(A.K1 - 1));
    A.b2lo[i] = fmaxf(u2 - h, 0.0f);
    A.b2hi[i] = fminf(u2 + h, (float)(A.K2 - 1));
}

__device__ __forceinline__ float div_at(const float* ph, const float* qh, const float* pv,
                                        const float* qv, long long i, int x, int y, int W, int H)
{
    float d = 0.0f;
    if (x + 1 < W) d += ph[i] - qh[i];
    if (x > 0) d -= ph[i - 1] - qh[i - 1];
    if (y + 1 < H) d += pv[i] - qv[i];
    if (y > 0) d -= pv[i - W] - qv[i - W];
    return d;
}

__global__ void flow_primal_kernel(FlowArgs A)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)A.H * A.W) return;
    const int y = (int)(i / A.W), x = (int)(i - (long long)y * A.W);
    const float tau = A.tau;
    const float uh1 = A.u1[i] - tau * div_at(A.ph1, A.qh1, A.pv1, A.qv1, i, x, y, A.W, A.H);
    const float uh2 = A.u2[i] - tau * div_at(A.ph2, A.qh2, A.pv2, A.qv2, i, x, y, A.W, A.H);
    const float q11 = A.q11[i], q12 = A.q12[i], q22 = A.q22[i];
    const float u01 = A.u01[i], u02 = A.u02[i];
    const float r1 = uh1 + tau * (q11 * u01 + q12 * u02 - A.L1[i]);
    const float r2 = uh2 + tau * (q12 * u01 + q22 * u02 - A.L2[i]);
    const float m11 = 1.0f + tau * q11, m12 = tau * q12, m22 = 1.0f + tau * q22;
    const float det = m11 * m22 - m12 * m12;
    const float v1 = (m22 * r1 - m12 * r2) / det;
    const float v2 = (m11 * r2 - m12 * r1) / det;
    A.un1[i] = fminf(fmaxf(v1, A.b1lo[i]), A.b1hi[i]);
    A.un2[i] = fminf(fmaxf(v2, A.b2lo[i]), A.b2hi[i]);
}

__global__ void flow_dual_kernel(FlowArgs A)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)A.H * A.W) return;
    const int y = (int)(i / A.W), x = (int)(i - (long long)y * A.W);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float* u = k == 0 ? A.u1 : A.u2;
        const float* un = k == 0 ? A.un1 : A.un2;
        float* ph = k == 0 ? A.ph1 : A.ph2;
        float* pv = k == 0 ? A.pv1 : A.pv2;
        float* qh = k == 0 ? A.qh1 : A.qh2;
        float* qv = k == 0 ? A.qv1 : A.qv2;
        const float ui = u[i], uni = un[i];
        if (x + 1 < A.W) {
            const float om = A.lambda_r * (float)A.wh[i];
            const float uj = u[i + 1], unj = un[i + 1];
            const float au = ui - uj;
            const float ext = (2.0f * uni - ui) - (2.0f * unj - uj);
            qh[i] = prox_conj_f(qh[i] + A.tau * au, om, 0.0f, A.bq, A.tau);
            ph[i] = prox_conj_f(ph[i] + A.sigma * ext, om, A.ap, A.bp, A.sigma);
        }
        if (y + 1 < A.H) {
            const float om = A.lambda_r * (float)A.wv[i];
            const float uj = u[i + A.W], unj = un[i + A.W];
            const float au = ui - uj;
            const float ext = (2.0f * uni - ui) - (2.0f * unj - uj);
            qv[i] = prox_conj_f(qv[i] + A.tau * au, om, 0.0f, A.bq, A.tau);
            pv[i] = prox_conj_f(pv[i] + A.sigma * ext, om, A.ap, A.bp, A.sigma);
        }
    }
}

__global__ void flow_export_kernel(FlowArgs A, float* __restrict__ d1, float* __restrict__ d2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)A.H * A.W) return;
    d1[i] = (float)A.lo1 + A.u1[i];
    d2[i] = (float)A.lo2 + A.u2[i];
}

unsigned blocks_of(const FlowArgs& a) { return (unsigned)(((long long)a.H * a.W + 255) / 256); }

}  // namespace

cudaError_t launch_flow_cost(const uint32_t* c1, const uint32_t* c2, int H, int W, int lo1, int K1,
                             int lo2, int K2, int maxc, uint8_t* p1, uint8_t* p2, cudaStream_t s)
{
    const long long px = (long long)H * W;
    const unsigned blocks = (unsigned)((px + kFlowWarps - 1) / kFlowWarps);
    flow_cost_kernel<<<blocks, kFlowWarps * 32, 0, s>>>(c1, c2, H, W, lo1, K1, lo2, K2, maxc, p1,
                                                        p2);
    return cudaGetLastError();
}

cudaError_t launch_flow_init(const FlowArgs& a, const uint16_t* lab1, const uint16_t* lab2,
                             cudaStream_t s)
{
    flow_init_kernel<<<blocks_of(a), 256, 0, s>>>(a, lab1, lab2);
    return cudaGetLastError();
}

cudaError_t launch_flow_lin(const FlowArgs& a, cudaStream_t s)
{
    flow_lin_kernel<<<blocks_of(a), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flow_iter(const FlowArgs& a, cudaStream_t s)
{
    flow_primal_kernel<<<blocks_of(a), 256, 0, s>>>(a);
    flow_dual_kernel<<<blocks_of(a), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flow_export(const FlowArgs& a, float* d1, float* d2, cudaStream_t s)
{
    flow_export_kernel<<<blocks_of(a), 256, 0, s>>>(a, d1, d2);
    return cudaGetLastError();
}

}  // namespace dm
