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

#include <algorithm>
#include <type_traits>
#include <utility>

#include "dm_internal.cuh"

namespace dm {
namespace {

constexpr int kTX = 32, kTY = 8;

// Programmatic dependent launch: an iteration kernel may be launched while the
// previous one drains; it waits for that grid (and its memory) before reading,
// and lets the next one launch once its own stores are issued.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// the cost samples: float32, uint16 or uint8 (the first that is set)
struct CostSrc {
    const uint8_t* c8;
    const uint16_t* c16;
    const float* cf;
};

__device__ __forceinline__ CostSrc cost_src(const PdArgs& A) { return {A.cost, A.cost16, A.costf}; }

__device__ __forceinline__ float cost_sample(const CostSrc& c, size_t i)
{
    if (c.cf != nullptr) return __ldg(c.cf + i);
    if (c.c16 != nullptr) return (float)__ldg(c.c16 + i);
    return (float)__ldg(c.c8 + i);
}

// The forward iteration and its reverse (below) recompute the same quantities
// and must take the same branches on them, so every rounding in these helpers
// is explicit (no contraction into fused multiply-adds left to the compiler).

// D_i(x): linear interpolation of the cost samples of pixel px with the argument
// clamped to [0, L-1]
__device__ __forceinline__ float interp(const CostSrc& c, int L, size_t px, float x)
{
    x = fminf(fmaxf(x, 0.0f), (float)(L - 1));
    int k = (int)floorf(x);
    if (k > L - 2) k = L - 2;
    if (k < 0) k = 0;
    const float t = __fsub_rn(x, (float)k);
    const float c0 = cost_sample(c, px * L + k);
    const float c1 = cost_sample(c, px * L + k + 1);
    return __fmaf_rn(t, __fsub_rn(c1, c0), c0);
}

__device__ __forceinline__ float alpha_of(const float* alpha_px, float alpha, int i)
{
    return alpha_px != nullptr ? __ldg(alpha_px + i) : alpha;
}

// The linearisation of Sec. 3.1 at u0: interpolated costs at u0 - h, u0, u0 + h
// and the two slopes before the convexity fix.
struct LinPx {
    float dm, d0, dp, s1, s2;
};

__device__ __forceinline__ LinPx lin_px(const CostSrc& c, int L, size_t px, float al, float u0,
                                        float h)
{
    LinPx r;
    r.d0 = interp(c, L, px, u0);
    r.dm = interp(c, L, px, __fsub_rn(u0, h));
    r.dp = interp(c, L, px, __fadd_rn(u0, h));
    r.s1 = __fdiv_rn(__fmul_rn(al, __fsub_rn(r.d0, r.dm)), h);
    r.s2 = __fdiv_rn(__fmul_rn(al, __fsub_rn(r.dp, r.d0)), h);
    return r;
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
__device__ __forceinline__ void lin_one(const PdArgs& A, int i)
{
    const float u0 = A.u[i];
    const LinPx l = lin_px(cost_src(A), A.L, i, alpha_of(A.alpha_px, A.alpha, i), u0, A.h);
    float s1 = l.s1, s2 = l.s2;
    if (s2 < s1) {
        s1 = 0.5f * __fadd_rn(s1, s2);
        s2 = s1;
    }
    A.u0[i] = u0;
    A.s1[i] = s1;
    A.s2[i] = s2;
    A.lo[i] = fmaxf(__fsub_rn(u0, A.h), 0.0f);
    A.hi[i] = fminf(__fadd_rn(u0, A.h), (float)(A.L - 1));
}

__global__ void linearise_kernel(const PdArgs A)
{
    wait_prior_grid();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.H * A.W) lin_one(A, i);
    allow_next_grid();
}

// prox of step * (omega r_{a,b})*: identity on |t| <= a omega, else shrink by
// b * step but not below a omega; then clamp to [-omega, omega] (Eq. pprox)
__device__ __forceinline__ float prox_conj(float t, float omega, float a, float b, float step)
{
    const float at = fabsf(t);
    const float ao = __fmul_rn(a, omega);
    float v = t;
    if (at > ao) v = copysignf(fmaxf(ao, __fmaf_rn(-b, step, at)), t);
    return fminf(fmaxf(v, -omega), omega);
}

// derivatives of prox_conj in t and in omega.  A tie goes to the branch whose
// derivative in t is zero: at |t| = a omega the value is the same on both
// branches, and for a omega = 0 the map is constant around t = 0.
__device__ __forceinline__ void prox_conj_d(float t, float omega, float a, float b, float step,
                                            float* dt, float* dom)
{
    const float at = fabsf(t);
    const float ao = __fmul_rn(a, omega);
    float v = t, d = 1.0f, g = 0.0f;
    if (at >= ao) {
        const float m = __fmaf_rn(-b, step, at);
        const float s = t > 0.0f ? 1.0f : (t < 0.0f ? -1.0f : 0.0f);
        if (m > ao) {
            v = s * m;
        } else {
            v = s * ao;
            d = 0.0f;
            g = s * a;
        }
    }
    if (v > omega) {
        d = 0.0f;
        g = 1.0f;
    } else if (v < -omega) {
        d = 0.0f;
        g = -1.0f;
    }
    *dt = d;
    *dom = g;
}

// arguments of the q and p proxes on the edge (i, j)
__device__ __forceinline__ float q_arg(float q, float tau, float ui, float uj)
{
    return __fmaf_rn(tau, __fsub_rn(ui, uj), q);
}

__device__ __forceinline__ float p_arg(float p, float sigma, float ui, float uni, float uj, float unj)
{
    const float ei = __fmaf_rn(2.0f, uni, -ui), ej = __fmaf_rn(2.0f, unj, -uj);
    return __fmaf_rn(sigma, __fsub_rn(ei, ej), p);
}

// u_hat = u - tau A^T (p - q) at pixel (x, y)
__device__ __forceinline__ float u_hat(const float* u, const float* ph, const float* pv,
                                       const float* qh, const float* qv, int W, int H, int x, int y,
                                       float tau)
{
    const int i = y * W + x;
    float div = 0.0f;
    if (x + 1 < W) div = __fadd_rn(div, __fsub_rn(ph[i], qh[i]));
    if (x > 0) div = __fsub_rn(div, __fsub_rn(ph[i - 1], qh[i - 1]));
    if (y + 1 < H) div = __fadd_rn(div, __fsub_rn(pv[i], qv[i]));
    if (y > 0) div = __fsub_rn(div, __fsub_rn(pv[i - W], qv[i - W]));
    return __fmaf_rn(-tau, div, u[i]);
}

// the same from values: (ph, qh) of the edges to the right (r) and from the
// left (l), (pv, qv) of the edges down (d) and from above (a); a flag is false
// where the image has no such edge.  Same operations in the same order.
__device__ __forceinline__ float u_hat_v(float u, bool r, float ph_r, float qh_r, bool l,
                                         float ph_l, float qh_l, bool d, float pv_d, float qv_d,
                                         bool a, float pv_a, float qv_a, float tau)
{
    float div = 0.0f;
    if (r) div = __fadd_rn(div, __fsub_rn(ph_r, qh_r));
    if (l) div = __fsub_rn(div, __fsub_rn(ph_l, qh_l));
    if (d) div = __fadd_rn(div, __fsub_rn(pv_d, qv_d));
    if (a) div = __fsub_rn(div, __fsub_rn(pv_a, qv_a));
    return __fmaf_rn(-tau, div, u);
}

// prox of tau times the linearised data term before the box clamp; *cs is the
// case taken: 0 above the kink, 1 below it, 2 at the kink u0
__device__ __forceinline__ float prox_lin(float uh, float u0, float s1, float s2, float tau, int* cs)
{
    const float ts1 = __fmul_rn(tau, s1), ts2 = __fmul_rn(tau, s2);
    if (uh > __fadd_rn(u0, ts2)) {
        *cs = 0;
        return __fsub_rn(uh, ts2);
    }
    if (uh < __fadd_rn(u0, ts1)) {
        *cs = 1;
        return __fsub_rn(uh, ts1);
    }
    *cs = 2;
    return u0;
}

// u+ at pixel (x, y) from the old state
__device__ __forceinline__ float u_step(const PdArgs& A, int x, int y)
{
    const int i = y * A.W + x;
    int cs;
    const float v = prox_lin(u_hat(A.u, A.ph, A.pv, A.qh, A.qv, A.W, A.H, x, y, A.tau), A.u0[i],
                             A.s1[i], A.s2[i], A.tau, &cs);
    return fminf(fmaxf(v, A.lo[i]), A.hi[i]);
}

// One TX x TY tile of the fused iteration: u+ on the tile and a one-pixel halo
// to the right and below (from the old p, q), then the tile's edges.  The whole
// CTA (TX * TY threads) calls it; there is no early exit, so a persistent loop
// may call it again after a barrier.
template <int TX, int TY>
__device__ __forceinline__ void pd_tile(const PdArgs& A, int x0, int y0, float (*s_un)[TX + 1],
                                        float (*s_u)[TX + 1])
{
    const int W = A.W, H = A.H;
    for (int t = threadIdx.x; t < (TX + 1) * (TY + 1); t += TX * TY) {
        const int lx = t % (TX + 1), ly = t / (TX + 1);
        const int x = x0 + lx, y = y0 + ly;
        if (x < W && y < H) {
            s_un[ly][lx] = u_step(A, x, y);
            s_u[ly][lx] = A.u[y * W + x];
        }
    }
    __syncthreads();
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int x = x0 + lx, y = y0 + ly;
    if (x < W && y < H) {
        const int i = y * W + x;
        const float ui = s_u[ly][lx];
        const float uni = s_un[ly][lx];
        A.u_new[i] = uni;
        if (x + 1 < W) {
            const float om = __fmul_rn(A.lambda_r, (float)A.wh[i]);
            const float uj = s_u[ly][lx + 1];
            A.qh2[i] = prox_conj(q_arg(A.qh[i], A.tau, ui, uj), om, 0.0f, A.bq, A.tau);
            A.ph2[i] = prox_conj(p_arg(A.ph[i], A.sigma, ui, uni, uj, s_un[ly][lx + 1]), om, A.ap,
                                 A.bp, A.sigma);
        }
        if (y + 1 < H) {
            const float om = __fmul_rn(A.lambda_r, (float)A.wv[i]);
            const float uj = s_u[ly + 1][lx];
            A.qv2[i] = prox_conj(q_arg(A.qv[i], A.tau, ui, uj), om, 0.0f, A.bq, A.tau);
            A.pv2[i] = prox_conj(p_arg(A.pv[i], A.sigma, ui, uni, uj, s_un[ly + 1][lx]), om, A.ap,
                                 A.bp, A.sigma);
        }
    }
}

__global__ void __launch_bounds__(kTX * kTY) pd_fused_kernel(const PdArgs A)
{
    __shared__ float s_un[kTY + 1][kTX + 1];  // u+ on the tile and its right/lower halo
    __shared__ float s_u[kTY + 1][kTX + 1];   // old u there
    wait_prior_grid();
    pd_tile<kTX, kTY>(A, blockIdx.x * kTX, blockIdx.y * kTY, s_un, s_u);
    allow_next_grid();
}

// --- the whole refinement in one cooperative launch -------------------------

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number k (1, 2, ...) over all CTAs of a cooperative launch: one
// arrival counter (zero at launch) that every CTA raises once per barrier and
// waits to reach k * gridDim.x (+ the test skew).  The wait is bounded by
// wait_ns of wall time; when it runs out, or another CTA has already given
// up, the CTA records kDevErrTimeout and the caller returns.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int32_t* err, int skew,
                                             long long wait_ns, unsigned k, int* s_go)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = k * gridDim.x + (unsigned)skew;
        const unsigned long long t0 = global_ns();
        int go = 1;
        while (ld_acquire(bar) < target) {
            if ((ld_relaxed(err) & kDevErrTimeout) != 0 ||
                global_ns() - t0 > (unsigned long long)wait_ns) {
                atomicOr(err, kDevErrTimeout);
                go = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *s_go = go;
    }
    __syncthreads();
    return *s_go != 0;
}

// Every iteration of dm_refine in one launch: the start (u from the labels or
// as given, zero duals), then per warp the linearisation and its iterations,
// each a sweep of the CTAs over the tiles of pd_tile followed by a grid
// barrier.  The arithmetic is pd_tile's and lin_one's, so the result is the
// one of the launch-per-iteration form bit for bit.
__global__ void __launch_bounds__(kTX * kTY) pd_run_kernel(const PdRunArgs R)
{
    __shared__ float s_un[kTY + 1][kTX + 1];
    __shared__ float s_u[kTY + 1][kTX + 1];
    __shared__ int s_go;
    const PdArgs& A0 = R.set[0];
    const int n = A0.H * A0.W;
    const int tiles_x = (A0.W + kTX - 1) / kTX;
    const int tiles = tiles_x * ((A0.H + kTY - 1) / kTY);
    const int stride = gridDim.x * blockDim.x;
    unsigned k = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (R.labels != nullptr) A0.u[i] = (float)R.labels[i];
        A0.ph[i] = A0.pv[i] = A0.qh[i] = A0.qv[i] = 0.0f;
        A0.ph2[i] = A0.pv2[i] = A0.qh2[i] = A0.qv2[i] = 0.0f;
    }
    if (!grid_barrier(R.bar, R.err, R.bar_skew, R.wait_ns, ++k, &s_go)) return;
    int cur = 0;
    const int base = R.iters / R.warps, extra = R.iters % R.warps;
    for (int w = 0; w < R.warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) lin_one(R.set[cur], i);
        if (!grid_barrier(R.bar, R.err, R.bar_skew, R.wait_ns, ++k, &s_go)) return;
        for (int it = 0; it < nit; ++it) {
            const PdArgs& A = R.set[cur];
            for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
                pd_tile<kTX, kTY>(A, (t % tiles_x) * kTX, (t / tiles_x) * kTY, s_un, s_u);
                __syncthreads();
            }
            if (!grid_barrier(R.bar, R.err, R.bar_skew, R.wait_ns, ++k, &s_go)) return;
            cur ^= 1;
        }
    }
}

// --- the whole refinement with the state in shared memory ---------------------

// shared-memory bytes of pd_res_kernel<NS>: nine float arrays (u twice, u0,
// s1, s2, ph, pv, qh, qv) and two weight byte arrays of NS entries each
__host__ __device__ constexpr size_t res_smem_bytes(int NS)
{
    return (size_t)NS * (9 * sizeof(float) + 2) + 16;
}

// the array strides pd_res_kernel is built for (the planner takes the smallest
// that holds the stored area)
constexpr int kResStrides[] = {1024, 2048, 3072, 4608, 5888};

// One CTA per region.  The CTA stores its region R and a margin of K pixels
// on each side that has a neighbouring region (the area E), and runs an epoch
// of up to K iterations on E alone: at step t (1..K) u+ is computed on E less
// t pixels on the left and upper margins and t - 1 on the right and lower ones
// (u_step's arithmetic, from values in shared memory), then q+, p+ on E less t
// on every margin (pd_tile's arithmetic).  Each step needs only values the
// previous step left valid, and after K steps R is exact.  Between epochs the
// regions exchange their K-wide borders through the workspace state set of
// the exchange's parity and a grid barrier; the other set still holds the
// previous exchange, which a CTA behind by one barrier may be reading.  Every
// warp of the refinement starts an epoch, whose first act is the
// linearisation of E.  Results equal pd_tile's bit for bit.
template <int NS>
__global__ void pd_res_kernel(const PdResArgs R)
{
    extern __shared__ float4 res_dyn[];
    __shared__ int s_go;
    const PdArgs& A = R.a;
    const int W = A.W, H = A.H, K = R.K, EW = R.EW;
    const int rxi = blockIdx.x % R.nx, ryi = blockIdx.x / R.nx;
    const int x0 = rxi * R.RW, y0 = ryi * R.RH;
    const int w_eff = min(R.RW, W - x0), h_eff = min(R.RH, H - y0);
    // E in image coordinates; a side shrinks during an epoch unless it is the
    // image's border
    const int ex0 = rxi > 0 ? x0 - K : 0, ey0 = ryi > 0 ? y0 - K : 0;
    const int ex1 = min(W, x0 + w_eff + (rxi + 1 < R.nx ? K : 0));
    const int ey1 = min(H, y0 + h_eff + (ryi + 1 < R.ny ? K : 0));
    const int ew = ex1 - ex0, eh = ey1 - ey0;
    const int shL = ex0 > 0, shR = ex1 < W, shU = ey0 > 0, shD = ey1 < H;
    // region R inside E
    const int rx0 = x0 - ex0, ry0 = y0 - ey0;
    // arrays of NS entries (NS >= EW * EH, a compile-time stride: every access
    // is one address plus a constant offset): the two u buffers, u0, s1, s2, the
    // duals, then the weights as bytes; cur says which u buffer is current
    float* const sb = reinterpret_cast<float*>(res_dyn);
    float* const su0 = sb + 2 * NS;
    float* const ss1 = sb + 3 * NS;
    float* const ss2 = sb + 4 * NS;
    float* const sph = sb + 5 * NS;
    float* const spv = sb + 6 * NS;
    float* const sqh = sb + 7 * NS;
    float* const sqv = sb + 8 * NS;
    uint8_t* const swh = reinterpret_cast<uint8_t*>(sb + 9 * NS);
    uint8_t* const swv = swh + NS;
    int cur = 0;
    const int TR = R.TR;
    const int tx = threadIdx.x % EW, ty = threadIdx.x / EW;
    const bool on = (int)threadIdx.x < EW * TR;
    const float tau = A.tau, sigma = A.sigma, h = A.h, top = (float)(A.L - 1);
    // the workspace state sets: 0 = (u, ph, pv, qh, qv), 1 = (u_new, ph2, ...)
    auto set_u = [&](int k) { return k ? A.u_new : A.u; };
    auto set_ph = [&](int k) { return k ? A.ph2 : A.ph; };
    auto set_pv = [&](int k) { return k ? A.pv2 : A.pv; };
    auto set_qh = [&](int k) { return k ? A.qh2 : A.qh; };
    auto set_qv = [&](int k) { return k ? A.qv2 : A.qv; };

    // start on all of E: u from the labels (or as given), zero duals
    if (on && tx < ew)
        for (int ey = ty; ey < eh; ey += TR) {
            const int p = ey * EW + tx, i = (ey0 + ey) * W + ex0 + tx;
            sb[p] = R.labels != nullptr ? (float)R.labels[i] : A.u[i];
            sph[p] = spv[p] = sqh[p] = sqv[p] = 0.0f;
            swh[p] = A.wh[i];
            swv[p] = A.wv[i];
        }
    __syncthreads();

    const CostSrc cs = cost_src(A);
    unsigned nbar = 0;   // grid barriers passed
    int nex = 0;         // exchanges done
    bool first = true;
    const int base = R.iters / R.warps, extra = R.iters % R.warps;
    for (int w = 0; w < R.warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        for (int done = 0; done < nit;) {
            const int steps = min(K, nit - done);
            float* const su = sb + cur * NS;   // the current u
            if (!first) {
                // exchange: R's K-wide border out, barrier, the margins of E in
                const int sp = nex & 1;
                if (on && tx >= rx0 && tx < rx0 + w_eff)
                    for (int ey = ry0 + ty; ey < ry0 + h_eff; ey += TR) {
                        const int rx = tx - rx0, ry = ey - ry0;
                        if (rx >= K && rx < w_eff - K && ry >= K && ry < h_eff - K) continue;
                        const int p = ey * EW + tx, i = (ey0 + ey) * W + ex0 + tx;
                        __stcg(set_u(sp) + i, su[p]);
                        __stcg(set_ph(sp) + i, sph[p]);
                        __stcg(set_pv(sp) + i, spv[p]);
                        __stcg(set_qh(sp) + i, sqh[p]);
                        __stcg(set_qv(sp) + i, sqv[p]);
                    }
                if (!grid_barrier(R.bar, R.err, R.wait_skew, R.wait_ns, ++nbar, &s_go)) return;
                if (on && tx < ew)
                    for (int ey = ty; ey < eh; ey += TR) {
                        if (tx >= rx0 && tx < rx0 + w_eff && ey >= ry0 && ey < ry0 + h_eff) continue;
                        const int p = ey * EW + tx, i = (ey0 + ey) * W + ex0 + tx;
                        su[p] = __ldcg(set_u(sp) + i);
                        sph[p] = __ldcg(set_ph(sp) + i);
                        spv[p] = __ldcg(set_pv(sp) + i);
                        sqh[p] = __ldcg(set_qh(sp) + i);
                        sqv[p] = __ldcg(set_qv(sp) + i);
                    }
                ++nex;
                __syncthreads();
            }
            first = false;
            if (done == 0) {
                // the warp's linearisation of E around its current u (lin_one)
                if (on && tx < ew)
                    for (int ey = ty; ey < eh; ey += TR) {
                        const int p = ey * EW + tx, i = (ey0 + ey) * W + ex0 + tx;
                        const float u0 = su[p];
                        const LinPx l = lin_px(cs, A.L, i, alpha_of(A.alpha_px, A.alpha, i), u0, h);
                        float s1 = l.s1, s2 = l.s2;
                        if (s2 < s1) {
                            s1 = 0.5f * __fadd_rn(s1, s2);
                            s2 = s1;
                        }
                        su0[p] = u0;
                        ss1[p] = s1;
                        ss2[p] = s2;
                    }
                __syncthreads();
            }
            // one step with the u buffers at constant offsets (CU: the current one)
            auto step = [&](auto cu_c, int t) {
                constexpr int CU = decltype(cu_c)::value;
                const float* const su = sb + CU * NS;
                float* const sun = sb + (1 - CU) * NS;
                // u+ on E less t (left, upper) and t - 1 (right, lower)
                {
                    const int xa = shL * t, xb = ew - shR * (t - 1);
                    const int ya = shU * t, yb = eh - shD * (t - 1);
                    if (on && tx >= xa && tx < xb)
                        for (int ey = ya + ty; ey < yb; ey += TR) {
                            const int p = ey * EW + tx, x = ex0 + tx, y = ey0 + ey;
                            const bool l = x > 0, a = y > 0;
                            const float uh = u_hat_v(su[p], x + 1 < W, sph[p], sqh[p], l,
                                                     l ? sph[p - 1] : 0.0f, l ? sqh[p - 1] : 0.0f,
                                                     y + 1 < H, spv[p], sqv[p], a,
                                                     a ? spv[p - EW] : 0.0f, a ? sqv[p - EW] : 0.0f,
                                                     tau);
                            const float u0 = su0[p];
                            int cse;
                            const float v = prox_lin(uh, u0, ss1[p], ss2[p], tau, &cse);
                            sun[p] = fminf(fmaxf(v, fmaxf(__fsub_rn(u0, h), 0.0f)),
                                           fminf(__fadd_rn(u0, h), top));
                        }
                }
                __syncthreads();
                // q+, p+ on E less t on every shrinking side
                {
                    const int xa = shL * t, xb = ew - shR * t;
                    const int ya = shU * t, yb = eh - shD * t;
                    if (on && tx >= xa && tx < xb)
                        for (int ey = ya + ty; ey < yb; ey += TR) {
                            const int p = ey * EW + tx, x = ex0 + tx, y = ey0 + ey;
                            const float ui = su[p], uni = sun[p];
                            if (x + 1 < W) {
                                const float om = __fmul_rn(A.lambda_r, (float)swh[p]);
                                const float uj = su[p + 1], unj = sun[p + 1];
                                sqh[p] = prox_conj(q_arg(sqh[p], tau, ui, uj), om, 0.0f, A.bq, tau);
                                sph[p] = prox_conj(p_arg(sph[p], sigma, ui, uni, uj, unj), om, A.ap,
                                                   A.bp, sigma);
                            }
                            if (y + 1 < H) {
                                const float om = __fmul_rn(A.lambda_r, (float)swv[p]);
                                const float uj = su[p + EW], unj = sun[p + EW];
                                sqv[p] = prox_conj(q_arg(sqv[p], tau, ui, uj), om, 0.0f, A.bq, tau);
                                spv[p] = prox_conj(p_arg(spv[p], sigma, ui, uni, uj, unj), om, A.ap,
                                                   A.bp, sigma);
                            }
                        }
                }
                __syncthreads();
            };
            for (int t = 1; t <= steps; ++t) {
                if (cur == 0) step(std::integral_constant<int, 0>{}, t);
                else step(std::integral_constant<int, 1>{}, t);
                cur ^= 1;
            }
            done += steps;
        }
    }
    // R's state into the set after the last exchange's (nobody reads it any
    // more), its linearisation into u0, s1, s2
    // with no exchange and a start given in set 0, another CTA may still be
    // reading its margin of that start
    if (nex == 0 && R.labels == nullptr && R.iters > 0 && gridDim.x > 1)
        if (!grid_barrier(R.bar, R.err, R.wait_skew, R.wait_ns, ++nbar, &s_go)) return;
    const int fs = nex & 1;
    const bool lin = R.iters > 0;
    const float* const su = sb + cur * NS;
    if (on && tx >= rx0 && tx < rx0 + w_eff)
        for (int ey = ry0 + ty; ey < ry0 + h_eff; ey += TR) {
            const int p = ey * EW + tx, i = (ey0 + ey) * W + ex0 + tx;
            set_u(fs)[i] = su[p];
            set_ph(fs)[i] = sph[p];
            set_pv(fs)[i] = spv[p];
            set_qh(fs)[i] = sqh[p];
            set_qv(fs)[i] = sqv[p];
            if (lin) {
                A.u0[i] = su0[p];
                A.s1[i] = ss1[p];
                A.s2[i] = ss2[p];
            }
        }
}


// --- batched forms over many pairs (one launch per iteration for all pairs) ---

// the pair whose range [start[p], start[p + 1]) holds t (start is ascending)
template <typename T>
__device__ __forceinline__ int pair_of(const T* start, int n, T t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// persistent: the CTAs stride over the tiles of all pairs
template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) pd_batch_kernel(const PdBatchArgs B)
{
    wait_prior_grid();
    __shared__ float s_un[TY + 1][TX + 1];
    __shared__ float s_u[TY + 1][TX + 1];
    for (int t = blockIdx.x; t < B.total_tiles; t += gridDim.x) {
        const int p = pair_of(B.tile_start, B.n, t);
        const PdArgs& A = B.descs[2 * p + B.parity];
        const int local = t - B.tile_start[p];
        const int tx = (A.W + TX - 1) / TX;
        pd_tile<TX, TY>(A, (local % tx) * TX, (local / tx) * TY, s_un, s_u);
        __syncthreads();
    }
    allow_next_grid();
}

// linearisation of every pixel of every pair (the current set of each pair)
__global__ void lin_batch_kernel(const PdBatchArgs B)
{
    wait_prior_grid();
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < B.total_px;
         g += (long long)gridDim.x * blockDim.x) {
        const int p = pair_of(B.px_start, B.n, g);
        lin_one(B.descs[2 * p + B.parity], (int)(g - B.px_start[p]));
    }
    allow_next_grid();
}

// u = labels in set 0, p = q = 0 in both sets, for every pair
__global__ void init_batch_kernel(const PdBatchArgs B)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < B.total_px;
         g += (long long)gridDim.x * blockDim.x) {
        const int p = pair_of(B.px_start, B.n, g);
        const int i = (int)(g - B.px_start[p]);
        const PdArgs& A = B.descs[2 * p];
        A.u[i] = (float)B.labels[p][i];
        A.ph[i] = A.pv[i] = A.qh[i] = A.qv[i] = 0.0f;
        A.ph2[i] = A.pv2[i] = A.qh2[i] = A.qv2[i] = 0.0f;
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
        acc += (double)alpha_of(A.alpha_px, A.alpha, i) * (double)interp(cost_src(A), A.L, i, u[i]);
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

// ---------------------------------------------------------------------------
// Reverse mode of the unrolled iteration (the differentiable refinement).
//
// Iteration k maps (u, p, q) to (u+, p+, q+) with
//   u+ = clamp_[lo,hi](prox_lin(u - tau A^T (p - q)))
//   q+ = prox_q(q + tau A u),   p+ = prox_p(p + sigma A (2u+ - u)).
// Given the adjoints (ub, pb, qb) of the outputs, the adjoints of the inputs are
//   tq = qb * dprox_q,  tp = pb * dprox_p                    (per edge)
//   ubar+ = ub + 2 sigma A^T tp,  uhb = ubar+ * dprox_lin     (per pixel)
//   ub' = uhb - sigma A^T tp + tau A^T tq
//   pb' = tp - tau A uhb,  qb' = tq + tau A uhb              (per edge)
// and the linearisation constants collect ubar+ on the branch the prox took.
// One kernel per iteration: a 32x8 tile computes tp, tq on its edges and on the
// edges entering it, then the pixel adjoints on the tile and a one-pixel halo
// to the right and below, then the dual adjoints of its own edges.

constexpr int kEX = kTX + 2, kEY = kTY + 2;  // edges owned by x0-1 .. x0+kTX, y0-1 .. y0+kTY
constexpr int kPX = kTX + 1, kPY = kTY + 1;  // pixels x0 .. x0+kTX, y0 .. y0+kTY

__global__ void __launch_bounds__(kTX * kTY) pd_adjoint_kernel(const AdjArgs A)
{
    wait_prior_grid();
    __shared__ float s_tph[kEY][kEX], s_tpv[kEY][kEX], s_tqh[kEY][kEX], s_tqv[kEY][kEX];
    __shared__ float s_uhb[kPY][kPX];
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int W = A.W, H = A.H;
    for (int t = threadIdx.x; t < kEX * kEY; t += kTX * kTY) {
        const int lx = t % kEX, ly = t / kEX;
        const int x = x0 - 1 + lx, y = y0 - 1 + ly;
        float tph = 0.0f, tpv = 0.0f, tqh = 0.0f, tqv = 0.0f;
        if (x >= 0 && y >= 0 && x < W && y < H) {
            const int i = y * W + x;
            const float ui = A.u[i], uni = A.un[i];
            float gl = 0.0f, d, g;
            if (x + 1 < W) {
                const float w = (float)A.wh[i];
                const float om = __fmul_rn(A.lambda_r, w);
                const float uj = A.u[i + 1];
                prox_conj_d(q_arg(A.qh[i], A.tau, ui, uj), om, 0.0f, A.bq, A.tau, &d, &g);
                const float bq = A.qhb[i];
                tqh = bq * d;
                gl += bq * g * w;
                prox_conj_d(p_arg(A.ph[i], A.sigma, ui, uni, uj, A.un[i + 1]), om, A.ap, A.bp,
                            A.sigma, &d, &g);
                const float bp = A.phb[i];
                tph = bp * d;
                gl += bp * g * w;
            }
            if (y + 1 < H) {
                const float w = (float)A.wv[i];
                const float om = __fmul_rn(A.lambda_r, w);
                const float uj = A.u[i + W];
                prox_conj_d(q_arg(A.qv[i], A.tau, ui, uj), om, 0.0f, A.bq, A.tau, &d, &g);
                const float bq = A.qvb[i];
                tqv = bq * d;
                gl += bq * g * w;
                prox_conj_d(p_arg(A.pv[i], A.sigma, ui, uni, uj, A.un[i + W]), om, A.ap, A.bp,
                            A.sigma, &d, &g);
                const float bp = A.pvb[i];
                tpv = bp * d;
                gl += bp * g * w;
            }
            if (lx >= 1 && lx <= kTX && ly >= 1 && ly <= kTY) A.glam[i] += gl;
        }
        s_tph[ly][lx] = tph;
        s_tpv[ly][lx] = tpv;
        s_tqh[ly][lx] = tqh;
        s_tqv[ly][lx] = tqv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kPX * kPY; t += kTX * kTY) {
        const int lx = t % kPX, ly = t / kPX;
        const int x = x0 + lx, y = y0 + ly;
        float uhb = 0.0f;
        if (x < W && y < H) {
            const int i = y * W + x;
            const int ex = lx + 1, ey = ly + 1;
            const float atp = s_tph[ey][ex] - s_tph[ey][ex - 1] + s_tpv[ey][ex] - s_tpv[ey - 1][ex];
            const float atq = s_tqh[ey][ex] - s_tqh[ey][ex - 1] + s_tqv[ey][ex] - s_tqv[ey - 1][ex];
            const float wbar = A.sigma * atp;
            const float unb = A.ub[i] + 2.0f * wbar;
            const float u0 = A.u0[i];
            int cs;
            const float v = prox_lin(u_hat(A.u, A.ph, A.pv, A.qh, A.qv, W, H, x, y, A.tau), u0,
                                     A.s1[i], A.s2[i], A.tau, &cs);
            float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
            if (v < A.lo[i]) {
                if (__fsub_rn(u0, A.h) > 0.0f) g0 = unb;      // lo = u0 - h
            } else if (v > A.hi[i]) {
                if (__fadd_rn(u0, A.h) < (float)(A.L - 1)) g0 = unb;  // hi = u0 + h
            } else if (cs == 0) {
                uhb = unb;
                g2 = -A.tau * unb;
            } else if (cs == 1) {
                uhb = unb;
                g1 = -A.tau * unb;
            } else {
                g0 = unb;
            }
            if (lx < kTX && ly < kTY) {
                A.ub2[i] = uhb - wbar + A.tau * atq;
                A.gu0[i] += g0;
                A.gs1[i] += g1;
                A.gs2[i] += g2;
            }
        }
        s_uhb[ly][lx] = uhb;
    }
    __syncthreads();
    const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) return;
    const int i = y * W + x;
    const float uhb = s_uhb[ly][lx];
    float phb = 0.0f, qhb = 0.0f, pvb = 0.0f, qvb = 0.0f;
    if (x + 1 < W) {
        const float d = A.tau * (uhb - s_uhb[ly][lx + 1]);
        phb = s_tph[ly + 1][lx + 1] - d;
        qhb = s_tqh[ly + 1][lx + 1] + d;
    }
    if (y + 1 < H) {
        const float d = A.tau * (uhb - s_uhb[ly + 1][lx]);
        pvb = s_tpv[ly + 1][lx + 1] - d;
        qvb = s_tqv[ly + 1][lx + 1] + d;
    }
    A.phb2[i] = phb;
    A.qhb2[i] = qhb;
    A.pvb2[i] = pvb;
    A.qvb2[i] = qvb;
    allow_next_grid();
}

// d D_i(x) / dx of the clamped interpolation (zero outside [0, L-1])
__device__ __forceinline__ float interp_dx(const CostSrc& c, int L, size_t px, float x)
{
    if (x < 0.0f || x > (float)(L - 1)) return 0.0f;
    int k = (int)floorf(x);
    if (k > L - 2) k = L - 2;
    return cost_sample(c, px * L + k + 1) - cost_sample(c, px * L + k);
}

// g += w * d D_i(x) / d c_i
__device__ __forceinline__ void interp_dc(float* g, int L, float x, float w)
{
    x = fminf(fmaxf(x, 0.0f), (float)(L - 1));
    int k = (int)floorf(x);
    if (k > L - 2) k = L - 2;
    if (k < 0) k = 0;
    const float t = __fsub_rn(x, (float)k);
    g[k] += w * (1.0f - t);
    g[k + 1] += w * t;
}

// Reverse of the linearisation at a warp start: the slope adjoints go through
// the convexity fix into the data weight, the cost samples and the point u0;
// the accumulators are cleared for the previous warp.
__global__ void lin_adjoint_kernel(const LinAdjArgs A)
{
    wait_prior_grid();
    const int n = A.H * A.W;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float u0 = A.u0[i], h = A.h;
    const float al = alpha_of(A.alpha_px, A.alpha, i);
    const CostSrc cs{A.cost, A.cost16, A.costf};
    const LinPx l = lin_px(cs, A.L, i, al, u0, h);
    float b1 = A.gs1[i], b2 = A.gs2[i];
    if (l.s2 < l.s1) b1 = b2 = 0.5f * (b1 + b2);
    const float um = __fsub_rn(u0, h), up = __fadd_rn(u0, h);
    if (A.galpha != nullptr) A.galpha[i] += (b1 * (l.d0 - l.dm) + b2 * (l.dp - l.d0)) / h;
    if (A.gcost != nullptr) {
        float* g = A.gcost + (size_t)i * A.L;
        interp_dc(g, A.L, u0, al / h * (b1 - b2));
        interp_dc(g, A.L, um, -al / h * b1);
        interp_dc(g, A.L, up, al / h * b2);
    }
    const float x0 = interp_dx(cs, A.L, i, u0);
    const float xm = interp_dx(cs, A.L, i, um);
    const float xp = interp_dx(cs, A.L, i, up);
    A.ub[i] += A.gu0[i] + al / h * (b1 * (x0 - xm) + b2 * (xp - x0));
    A.gu0[i] = 0.0f;
    A.gs1[i] = 0.0f;
    A.gs2[i] = 0.0f;
    allow_next_grid();
}

// ---------------------------------------------------------------------------
// Forward mode (tangents) of the unrolled iteration, on the branches the
// forward takes: the directional derivative of u in a direction (dc, dalpha,
// dlambda, du0).  It is the transpose of the reverse mode above; the pair
// satisfies <gu, J v> = <J^T gu, v> on any trajectory.

// linearisation of a warp and its tangent (u0 = u at the warp start)
__global__ void lin_jvp_kernel(const JvpArgs J)
{
    wait_prior_grid();
    const PdArgs& A = J.f;
    const int n = A.H * A.W;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float u0 = A.u[i], du0 = J.du[i], h = A.h;
    const float al = alpha_of(A.alpha_px, A.alpha, i);
    const float dal = J.dalpha != nullptr ? J.dalpha[i] : 0.0f;
    const CostSrc cs = cost_src(A);
    const LinPx l = lin_px(cs, A.L, i, al, u0, h);
    const float um = __fsub_rn(u0, h), up = __fadd_rn(u0, h);
    float dd0 = interp_dx(cs, A.L, i, u0) * du0;
    float ddm = interp_dx(cs, A.L, i, um) * du0;
    float ddp = interp_dx(cs, A.L, i, up) * du0;
    if (J.dcost != nullptr) {
        const CostSrc dc{nullptr, nullptr, J.dcost};
        dd0 += interp(dc, A.L, i, u0);
        ddm += interp(dc, A.L, i, um);
        ddp += interp(dc, A.L, i, up);
    }
    float s1 = l.s1, s2 = l.s2;
    float ds1 = (dal * (l.d0 - l.dm) + al * (dd0 - ddm)) / h;
    float ds2 = (dal * (l.dp - l.d0) + al * (ddp - dd0)) / h;
    if (s2 < s1) {
        s1 = 0.5f * __fadd_rn(s1, s2);
        s2 = s1;
        ds1 = ds2 = 0.5f * (ds1 + ds2);
    }
    A.u0[i] = u0;
    A.s1[i] = s1;
    A.s2[i] = s2;
    A.lo[i] = fmaxf(um, 0.0f);
    A.hi[i] = fminf(up, (float)(A.L - 1));
    J.du0[i] = du0;
    J.ds1[i] = ds1;
    J.ds2[i] = ds2;
    J.dlo[i] = um > 0.0f ? du0 : 0.0f;
    J.dhi[i] = up < (float)(A.L - 1) ? du0 : 0.0f;
    allow_next_grid();
}

__global__ void __launch_bounds__(kTX * kTY) pd_jvp_kernel(const JvpArgs J)
{
    wait_prior_grid();
    const PdArgs& A = J.f;
    __shared__ float s_un[kTY + 1][kTX + 1], s_u[kTY + 1][kTX + 1];
    __shared__ float s_dun[kTY + 1][kTX + 1], s_du[kTY + 1][kTX + 1];
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int W = A.W, H = A.H;
    for (int t = threadIdx.x; t < (kTX + 1) * (kTY + 1); t += kTX * kTY) {
        const int lx = t % (kTX + 1), ly = t / (kTX + 1);
        const int x = x0 + lx, y = y0 + ly;
        if (x < W && y < H) {
            const int i = y * W + x;
            int cs;
            const float v = prox_lin(u_hat(A.u, A.ph, A.pv, A.qh, A.qv, W, H, x, y, A.tau), A.u0[i],
                                     A.s1[i], A.s2[i], A.tau, &cs);
            float ddiv = 0.0f;
            if (x + 1 < W) ddiv += J.dph[i] - J.dqh[i];
            if (x > 0) ddiv -= J.dph[i - 1] - J.dqh[i - 1];
            if (y + 1 < H) ddiv += J.dpv[i] - J.dqv[i];
            if (y > 0) ddiv -= J.dpv[i - W] - J.dqv[i - W];
            const float duh = J.du[i] - A.tau * ddiv;
            const float un = fminf(fmaxf(v, A.lo[i]), A.hi[i]);
            float dun;
            if (v < A.lo[i])
                dun = J.dlo[i];
            else if (v > A.hi[i])
                dun = J.dhi[i];
            else
                dun = cs == 0 ? duh - A.tau * J.ds2[i] : (cs == 1 ? duh - A.tau * J.ds1[i] : J.du0[i]);
            s_un[ly][lx] = un;
            s_u[ly][lx] = A.u[i];
            s_dun[ly][lx] = dun;
            s_du[ly][lx] = J.du[i];
        }
    }
    __syncthreads();
    const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) return;
    const int i = y * W + x;
    const float ui = s_u[ly][lx], uni = s_un[ly][lx];
    const float dui = s_du[ly][lx], deni = 2.0f * s_dun[ly][lx] - dui;
    A.u_new[i] = uni;
    J.du2[i] = s_dun[ly][lx];
    float d, g;
    if (x + 1 < W) {
        const float w = (float)A.wh[i];
        const float om = __fmul_rn(A.lambda_r, w), dom = J.dlambda * w;
        const float uj = s_u[ly][lx + 1], duj = s_du[ly][lx + 1];
        const float tq = q_arg(A.qh[i], A.tau, ui, uj);
        A.qh2[i] = prox_conj(tq, om, 0.0f, A.bq, A.tau);
        prox_conj_d(tq, om, 0.0f, A.bq, A.tau, &d, &g);
        J.dqh2[i] = d * (J.dqh[i] + A.tau * (dui - duj)) + g * dom;
        const float tp = p_arg(A.ph[i], A.sigma, ui, uni, uj, s_un[ly][lx + 1]);
        A.ph2[i] = prox_conj(tp, om, A.ap, A.bp, A.sigma);
        prox_conj_d(tp, om, A.ap, A.bp, A.sigma, &d, &g);
        const float denj = 2.0f * s_dun[ly][lx + 1] - duj;
        J.dph2[i] = d * (J.dph[i] + A.sigma * (deni - denj)) + g * dom;
    } else {
        J.dqh2[i] = 0.0f;
        J.dph2[i] = 0.0f;
    }
    if (y + 1 < H) {
        const float w = (float)A.wv[i];
        const float om = __fmul_rn(A.lambda_r, w), dom = J.dlambda * w;
        const float uj = s_u[ly + 1][lx], duj = s_du[ly + 1][lx];
        const float tq = q_arg(A.qv[i], A.tau, ui, uj);
        A.qv2[i] = prox_conj(tq, om, 0.0f, A.bq, A.tau);
        prox_conj_d(tq, om, 0.0f, A.bq, A.tau, &d, &g);
        J.dqv2[i] = d * (J.dqv[i] + A.tau * (dui - duj)) + g * dom;
        const float tp = p_arg(A.pv[i], A.sigma, ui, uni, uj, s_un[ly + 1][lx]);
        A.pv2[i] = prox_conj(tp, om, A.ap, A.bp, A.sigma);
        prox_conj_d(tp, om, A.ap, A.bp, A.sigma, &d, &g);
        const float denj = 2.0f * s_dun[ly + 1][lx] - duj;
        J.dpv2[i] = d * (J.dpv[i] + A.sigma * (deni - denj)) + g * dom;
    } else {
        J.dqv2[i] = 0.0f;
        J.dpv2[i] = 0.0f;
    }
    allow_next_grid();
}

constexpr int kSumThreads = 256, kSumBlocks = 152;

// fixed-order sum of a float array in double: per-block partials, then one block
__global__ void sum_partial_kernel(const float* __restrict__ x, int n, double* __restrict__ partial)
{
    __shared__ double sh[kSumThreads];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc += (double)x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kSumThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void sum_final_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += partial[b];
        *out = acc;
    }
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

// launch with programmatic stream serialisation (see wait_prior_grid)
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t s, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

cudaError_t launch_linearise(const PdArgs& a, cudaStream_t s)
{
    const int n = a.H * a.W;
    return launch_pdl(linearise_kernel, dim3((n + 255) / 256), dim3(256), s, a);
}

cudaError_t launch_pd_iter(const PdArgs& a, cudaStream_t s)
{
    dim3 grd((a.W + kTX - 1) / kTX, (a.H + kTY - 1) / kTY);
    return launch_pdl(pd_fused_kernel, grd, dim3(kTX * kTY), s, a);
}

// CTAs of pd_run_kernel: as many as can be resident at once (the cooperative
// launch checks it), at most one per tile; CTA b takes the tiles b, b + grid,
// ..., so the SMs' tile counts differ by at most one CTA's extra tile
int pd_run_grid(int H, int W)
{
    static int max_ctas = 0;
    if (max_ctas == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pd_run_kernel, kTX * kTY, 0) !=
                cudaSuccess)
            return 0;
        max_ctas = sms * per_sm;
    }
    const int tiles = ((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY);
    return tiles < max_ctas ? tiles : max_ctas;
}

cudaError_t launch_pd_run(const PdRunArgs& r, cudaStream_t s)
{
    const int grid = pd_run_grid(r.set[0].H, r.set[0].W);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTX * kTY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pd_run_kernel, r);
}

// Regions of pd_res_kernel: at most one per SM and about 1024 pixels or more
// each; among the region grids nx x ny that fit, the one with the smallest
// region (then the shortest boundary).  The margin K is kResK, or less where a
// region is thinner.  False when the stored area does not fit in shared memory
// (or one of its rows in one CTA): the caller takes pd_run_kernel instead.
constexpr int kResK = 5;

bool pd_res_plan(int H, int W, PdResPlan* plan)
{
    static int sms = 0, max_smem = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess) {
            sms = 0;
            return false;
        }
    }
    const long long px = (long long)H * W;
    const int want = (int)std::min<long long>(sms, std::max<long long>(1, (px + 1023) / 1024));
    long long best_area = -1, best_per = 0;
    // first only grids whose split axes keep regions at least kResK wide
    for (int thin = 0; thin < 2 && best_area < 0; ++thin)
        for (int nx = 1; nx <= std::min(W, want); ++nx) {
            const int ny0 = std::min(H, want / nx);
            if (ny0 < 1) break;
            const int RW = (W + nx - 1) / nx, RH = (H + ny0 - 1) / ny0;
            if (!thin && ((nx > 1 && RW < kResK) || (ny0 > 1 && RH < kResK))) continue;
            const long long area = (long long)RW * RH, per = RW + RH;
            if (best_area < 0 || area < best_area || (area == best_area && per < best_per)) {
                best_area = area;
                best_per = per;
                plan->RW = RW;
                plan->RH = RH;
            }
        }
    if (best_area < 0) return false;
    plan->nx = (W + plan->RW - 1) / plan->RW;
    plan->ny = (H + plan->RH - 1) / plan->RH;
    int K = kResK;
    if (plan->nx > 1) K = std::min(K, plan->RW);
    if (plan->ny > 1) K = std::min(K, plan->RH);
    plan->K = K;
    plan->EW = plan->RW + (plan->nx > 1 ? 2 * K : 0);
    plan->EH = plan->RH + (plan->ny > 1 ? 2 * K : 0);
    if (plan->EW > 1024) return false;
    plan->NS = 0;
    for (const int ns : kResStrides)
        if (ns >= plan->EW * plan->EH) {
            plan->NS = ns;
            break;
        }
    if (plan->NS == 0) return false;
    plan->smem = res_smem_bytes(plan->NS);
    if (plan->smem > (size_t)max_smem) return false;
    plan->TR = std::min(plan->EH, 1024 / plan->EW);
    plan->threads = (plan->EW * plan->TR + 31) / 32 * 32;
    return plan->nx * plan->ny <= sms;
}

int pd_res_result_set(int iters, int warps, int K)
{
    const int base = iters / warps, extra = iters % warps;
    int epochs = 0;
    for (int w = 0; w < warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        epochs += (nit + K - 1) / K;
    }
    return epochs > 1 ? (epochs - 1) & 1 : 0;
}

template <int NS>
cudaError_t launch_pd_res_t(const PdResArgs& r, const PdResPlan& plan, cudaStream_t s)
{
    static size_t smem_set = 0;   // the opt-in is raised once per larger size
    if (plan.smem > smem_set) {
        const cudaError_t e = cudaFuncSetAttribute(
            pd_res_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
        if (e != cudaSuccess) return e;
        smem_set = plan.smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.nx * plan.ny);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pd_res_kernel<NS>, r);
}

cudaError_t launch_pd_res(const PdResArgs& r, const PdResPlan& plan, cudaStream_t s)
{
    switch (plan.NS) {
        case 1024: return launch_pd_res_t<1024>(r, plan, s);
        case 2048: return launch_pd_res_t<2048>(r, plan, s);
        case 3072: return launch_pd_res_t<3072>(r, plan, s);
        case 4608: return launch_pd_res_t<4608>(r, plan, s);
        case 5888: return launch_pd_res_t<5888>(r, plan, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int TX, int TY>
cudaError_t launch_pd_batch_t(const PdBatchArgs& b, int grid, cudaStream_t s)
{
    return launch_pdl(pd_batch_kernel<TX, TY>, dim3(grid), dim3(TX * TY), s, b);
}

bool pd_tile_supported(int tx, int ty)
{
    return (tx == 32 && (ty == 4 || ty == 8 || ty == 16)) || (tx == 64 && (ty == 4 || ty == 8)) ||
           (tx == 16 && ty == 16);
}

cudaError_t launch_pd_batch(const PdBatchArgs& b, int tx, int ty, int grid, cudaStream_t s)
{
    if (tx == 32 && ty == 4) return launch_pd_batch_t<32, 4>(b, grid, s);
    if (tx == 32 && ty == 16) return launch_pd_batch_t<32, 16>(b, grid, s);
    if (tx == 64 && ty == 4) return launch_pd_batch_t<64, 4>(b, grid, s);
    if (tx == 64 && ty == 8) return launch_pd_batch_t<64, 8>(b, grid, s);
    if (tx == 16 && ty == 16) return launch_pd_batch_t<16, 16>(b, grid, s);
    return launch_pd_batch_t<32, 8>(b, grid, s);
}

cudaError_t launch_lin_batch(const PdBatchArgs& b, int grid, cudaStream_t s)
{
    return launch_pdl(lin_batch_kernel, dim3(grid), dim3(256), s, b);
}

cudaError_t launch_init_batch(const PdBatchArgs& b, int grid, cudaStream_t s)
{
    init_batch_kernel<<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_pd_adjoint(const AdjArgs& a, cudaStream_t s)
{
    dim3 grd((a.W + kTX - 1) / kTX, (a.H + kTY - 1) / kTY);
    return launch_pdl(pd_adjoint_kernel, grd, dim3(kTX * kTY), s, a);
}

cudaError_t launch_lin_adjoint(const LinAdjArgs& a, cudaStream_t s)
{
    const int n = a.H * a.W;
    return launch_pdl(lin_adjoint_kernel, dim3((n + 255) / 256), dim3(256), s, a);
}

cudaError_t launch_lin_jvp(const JvpArgs& a, cudaStream_t s)
{
    const int n = a.f.H * a.f.W;
    return launch_pdl(lin_jvp_kernel, dim3((n + 255) / 256), dim3(256), s, a);
}

cudaError_t launch_pd_jvp(const JvpArgs& a, cudaStream_t s)
{
    dim3 grd((a.f.W + kTX - 1) / kTX, (a.f.H + kTY - 1) / kTY);
    return launch_pdl(pd_jvp_kernel, grd, dim3(kTX * kTY), s, a);
}

// partial must hold kSumBlocks doubles
cudaError_t launch_sum_f32(const float* x, int n, double* partial, double* out, cudaStream_t s)
{
    sum_partial_kernel<<<kSumBlocks, kSumThreads, 0, s>>>(x, n, partial);
    sum_final_kernel<<<1, 32, 0, s>>>(partial, kSumBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_energy(const PdArgs& a, double eps, double delta, double C, double* partial,
                          int nblocks, cudaStream_t s)
{
    energy_kernel<<<nblocks, kEnergyThreads, 0, s>>>(a, eps, delta, C, partial);
    return cudaGetLastError();
}

}  // namespace dm
