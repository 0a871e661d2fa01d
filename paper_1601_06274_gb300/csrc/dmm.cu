// One pass of Dual MM (Alg. Dual_MM of arXiv 1601.06274) over all horizontal
// or all vertical chains, each chain minorised with the hierarchical minorant
// of App. A (Alg. Handshake).
//
// Work decomposition
//   * One CTA per chain (a row for the horizontal pass, a column for the
//     vertical pass); the chains are independent (Sec. 2.3: the minorants
//     decouple over chains).
//   * The hierarchy is walked level by level inside the CTA.  Level l holds
//     up to 2^l sub-chains ("segments"); each level has a sweep phase (one warp
//     per message sweep) and a Handshake phase (one warp per segment),
//     separated by __syncthreads.  A sweep recomputes only the messages whose
//     boundary message changed (Fig. hierarchical-msgs): a left child keeps the
//     left messages of its ancestors and sweeps from its right end, a right
//     child the reverse.
//   * Messages live in a positional scratch: fmsg[k] is the message entering
//     node k from the left, bmsg[k] the one entering from the right.  Sweeps
//     store every message they produce; a Handshake over (i, j) stores
//     fmsg[j] (the left boundary of the right child) and bmsg[i].  At the end
//     node k keeps theta_k + fmsg[k] + bmsg[k].
//   * Labels are spread over the 32 lanes of a warp, LPT consecutive labels per
//     lane.  A message Msg(a)(x') = min_x a(x) + omega r(|x - x'|) is computed
//     in O(L): r is truncated at C, so only label distances d <= R with
//     omega r(d) < omega C can beat the cap min(a) + omega C.  Neighbouring
//     labels in other lanes are fetched with shuffles, the cap with one
//     warp-wide REDUX min.
//   * All arithmetic is int32 without normalisation; the host admits a cost
//     volume only if (max cost + 4 omega C) times the chain length stays below
//     2^30, so no value approaches the int32 range.

#include "dm_internal.cuh"

namespace dm {
namespace {

constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;

// cost sample i of the uint8 or uint16 volume
__device__ __forceinline__ int cost_of(const DmmArgs& A, size_t i)
{
    return A.cost16 != nullptr ? (int)__ldg(A.cost16 + i) : (int)__ldg(A.cost + i);
}

// value of label index (lane * LPT + j + off) for a compile-time off in [-R, LPT-1+R]
template <int LPT, int OFF>
__device__ __forceinline__ int neighbour(const int (&a)[LPT], int lane)
{
    constexpr int lo = (OFF >= 0) ? OFF / LPT : -((-OFF + LPT - 1) / LPT);  // floor(OFF / LPT)
    constexpr int loc = OFF - lo * LPT;
    if constexpr (lo == 0) {
        return a[loc];
    } else if constexpr (lo < 0) {
        const int v = __shfl_up_sync(kFull, a[loc], -lo);
        return (lane + lo >= 0) ? v : kInf;
    } else {
        const int v = __shfl_down_sync(kFull, a[loc], lo);
        return (lane + lo <= 31) ? v : kInf;
    }
}

// ext[IDX + R] = value of label index (lane * LPT + IDX), IDX in [-R, LPT + R)
template <int LPT, int R, int IDX>
__device__ __forceinline__ void fill_ext(const int (&a)[LPT], int (&ext)[LPT + 2 * R], int lane)
{
    if constexpr (IDX < LPT + R) {
        ext[IDX + R] = neighbour<LPT, IDX>(a, lane);
        fill_ext<LPT, R, IDX + 1>(a, ext, lane);
    }
}

// out = Msg(a) for the edge with penalty taps `tap` (T_1..T_R, P2 at kTapP2).
// Padding labels (>= L) of `a` are forced to kInf first when PAD.
template <int LPT, int R, bool PAD>
__device__ __forceinline__ void msg(int (&a)[LPT], int (&out)[LPT], const int* tap, int lane,
                                    int L)
{
    if constexpr (PAD) {
#pragma unroll
        for (int j = 0; j < LPT; ++j)
            if (lane * LPT + j >= L) a[j] = kInf;
    }
    int m = a[0];
#pragma unroll
    for (int j = 1; j < LPT; ++j) m = min(m, a[j]);
    m = __reduce_min_sync(kFull, m);
    int ext[LPT + 2 * R];
    fill_ext<LPT, R, -R>(a, ext, lane);
    int res[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) res[j] = a[j];
#pragma unroll
    for (int d = 1; d <= R; ++d) {
        const int T = tap[d - 1];
#pragma unroll
        for (int j = 0; j < LPT; ++j) res[j] = min(res[j], min(ext[j - d + R], ext[j + d + R]) + T);
    }
    const int cap = m + tap[kTapP2];
#pragma unroll
    for (int j = 0; j < LPT; ++j) out[j] = min(res[j], cap);
}

struct Chain {
    int which, W, L, KP, n;
    int c;  // chain index
    __device__ __forceinline__ size_t pix(int k) const
    {
        return which == 0 ? (size_t)c * W + k : (size_t)k * W + c;
    }
};

template <int LPT>
__device__ __forceinline__ void load_theta(const DmmArgs& A, const Chain& ch, int k, int lane,
                                           int (&th)[LPT])
{
    const size_t base = ch.pix(k) * (size_t)ch.L + (size_t)lane * LPT;
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int l = lane * LPT + j;
        int v = kInf;
        if (l < ch.L) {
            v = __ldg(A.lam_in + base + j);
            if (ch.which == 0) v += cost_of(A, base + j);
        }
        th[j] = v;
    }
}

template <int LPT>
__device__ __forceinline__ void load_msg(const int32_t* buf, int lane, int (&m)[LPT])
{
    const int32_t* p = buf + lane * LPT;
    if constexpr (LPT == 4) {
        const int4 v = *reinterpret_cast<const int4*>(p);
        m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
    } else if constexpr (LPT == 2) {
        const int2 v = *reinterpret_cast<const int2*>(p);
        m[0] = v.x; m[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < LPT; ++j) m[j] = p[j];
    }
}

template <int LPT>
__device__ __forceinline__ void store_msg(int32_t* buf, int lane, const int (&m)[LPT])
{
    int32_t* p = buf + lane * LPT;
    if constexpr (LPT == 4) {
        *reinterpret_cast<int4*>(p) = make_int4(m[0], m[1], m[2], m[3]);
    } else if constexpr (LPT == 2) {
        *reinterpret_cast<int2*>(p) = make_int2(m[0], m[1]);
    } else {
#pragma unroll
        for (int j = 0; j < LPT; ++j) p[j] = m[j];
    }
}

__device__ __forceinline__ const int* edge_taps(const DmmArgs& A, const Chain& ch, int k)
{
    // edge between chain nodes k and k+1 is stored at node k
    const int om = __ldg(A.wedge + ch.pix(k));
    const int* tap = A.taps + om * kTapW;
    if (__ldg(tap + kTapValid) == 0) atomicOr(A.err, kDevErrBadOmega);
    return tap;
}

// Segment `s` of level `level` of the split tree of [0, n); the left part of
// a split keeps ceil(len / 2) nodes.  Returns false when the segment does not
// exist (an ancestor was already a single node).
__device__ __forceinline__ bool segment(int n, int level, int s, int& a, int& b)
{
    a = 0;
    b = n - 1;
    for (int bit = level - 1; bit >= 0; --bit) {
        const int len = b - a + 1;
        if (len == 1) return false;
        const int i = a + ((len + 1) >> 1) - 1;
        if ((s >> bit) & 1) a = i + 1;
        else b = i;
    }
    return true;
}

template <int LPT, int R, bool PAD>
__global__ void __launch_bounds__(kWarps * 32) dmm_pass_kernel(const DmmArgs A)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Chain ch;
    ch.which = A.which;
    ch.W = A.W;
    ch.L = A.L;
    ch.KP = A.KP;
    ch.n = A.which == 0 ? A.W : A.H;
    ch.c = blockIdx.x;
    const int n = ch.n;
    int32_t* F = A.fmsg + (size_t)ch.c * n * A.KP;
    int32_t* B = A.bmsg + (size_t)ch.c * n * A.KP;

    // zero boundary messages at both chain ends
    if (warp == 0) {
        for (int l = lane; l < A.KP; l += 32) {
            F[l] = 0;
            B[(size_t)(n - 1) * A.KP + l] = 0;
        }
    }
    __syncthreads();

    int levels = 0;
    while ((1 << levels) < n) ++levels;  // ceil(log2 n)

    for (int level = 0; level < levels; ++level) {
        // ---- sweep phase ------------------------------------------------------
        const int nseg = 1 << level;
        const int ntask = level == 0 ? 2 : nseg;
        for (int t = warp; t < ntask; t += kWarps) {
            const int s = level == 0 ? 0 : t;
            int a, b;
            if (!segment(n, level, s, a, b) || b <= a) continue;
            const int i = a + ((b - a + 2) >> 1) - 1;
            const int j = i + 1;
            const bool fwd = level == 0 ? (t == 0) : ((s & 1) == 1);  // right children sweep forward
            int msgv[LPT], th[LPT], x[LPT];
            if (fwd) {
                if (i == a) continue;
                load_msg<LPT>(F + (size_t)a * A.KP, lane, msgv);
                for (int k = a; k < i; ++k) {
                    load_theta<LPT>(A, ch, k, lane, th);
                    const int* tap = edge_taps(A, ch, k);
#pragma unroll
                    for (int q = 0; q < LPT; ++q) x[q] = th[q] + msgv[q];
                    msg<LPT, R, PAD>(x, msgv, tap, lane, A.L);
                    store_msg<LPT>(F + (size_t)(k + 1) * A.KP, lane, msgv);
                }
            } else {
                if (b == j) continue;
                load_msg<LPT>(B + (size_t)b * A.KP, lane, msgv);
                for (int k = b; k > j; --k) {
                    load_theta<LPT>(A, ch, k, lane, th);
                    const int* tap = edge_taps(A, ch, k - 1);
#pragma unroll
                    for (int q = 0; q < LPT; ++q) x[q] = th[q] + msgv[q];
                    msg<LPT, R, PAD>(x, msgv, tap, lane, A.L);
                    store_msg<LPT>(B + (size_t)(k - 1) * A.KP, lane, msgv);
                }
            }
        }
        __syncthreads();
        // ---- Handshake phase --------------------------------------------------
        for (int s = warp; s < nseg; s += kWarps) {
            int a, b;
            if (!segment(n, level, s, a, b) || b <= a) continue;
            const int i = a + ((b - a + 2) >> 1) - 1;
            const int j = i + 1;
            int Fi[LPT], Bj[LPT], thi[LPT], thj[LPT], x[LPT], phi_ji[LPT], phi_ij[LPT];
            load_msg<LPT>(F + (size_t)i * A.KP, lane, Fi);
            load_msg<LPT>(B + (size_t)j * A.KP, lane, Bj);
            load_theta<LPT>(A, ch, i, lane, thi);
            load_theta<LPT>(A, ch, j, lane, thj);
            const int* tap = edge_taps(A, ch, i);
#pragma unroll
            for (int q = 0; q < LPT; ++q) x[q] = thj[q] + Bj[q];
            msg<LPT, R, PAD>(x, phi_ji, tap, lane, A.L);           // message j -> i
#pragma unroll
            for (int q = 0; q < LPT; ++q)                           // half of the min-marginal at i
                x[q] = ((Fi[q] + thi[q] + phi_ji[q]) >> 1) - phi_ji[q];
            msg<LPT, R, PAD>(x, phi_ij, tap, lane, A.L);           // share it to the right
#pragma unroll
            for (int q = 0; q < LPT; ++q) x[q] = -phi_ij[q];
            msg<LPT, R, true>(x, phi_ji, tap, lane, A.L);          // bounce back the rest
            store_msg<LPT>(F + (size_t)j * A.KP, lane, phi_ij);
            store_msg<LPT>(B + (size_t)i * A.KP, lane, phi_ji);
        }
        __syncthreads();
    }

    // ---- every node keeps its whole remaining min-marginal -----------------------
    long long lb_acc = 0;
    for (int k = warp; k < n; k += kWarps) {
        int fk[LPT], bk[LPT];
        load_msg<LPT>(F + (size_t)k * A.KP, lane, fk);
        load_msg<LPT>(B + (size_t)k * A.KP, lane, bk);
        const size_t pix = ch.pix(k);
        const size_t base = pix * (size_t)A.L + (size_t)lane * LPT;
        int best = kInf, arg = 0x7fffffff;
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int l = lane * LPT + j;
            if (l < A.L) {
                const int inl = __ldg(A.lam_in + base + j);
                int out = fk[j] + bk[j];                  // lambda_out = theta + F + B - lam_in
                if (A.which == 0) out += cost_of(A, base + j);
                A.lam_out[base + j] = out;
                const int nu = out + inl;                 // lambda_h + lambda_v
                if (nu < best) {
                    best = nu;
                    arg = l;
                }
            }
        }
        if (A.labels != nullptr || A.lb != nullptr) {
            const int m = __reduce_min_sync(kFull, best);
            if (A.labels != nullptr) {
                const int cand = (best == m) ? arg : 0x7fffffff;
                const int am = __reduce_min_sync(kFull, cand);
                if (lane == 0) A.labels[pix] = (uint16_t)am;
            }
            lb_acc += m;
        }
    }
    if (A.lb != nullptr && lane == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(A.lb), (unsigned long long)lb_acc);
}

template <int LPT, int R>
cudaError_t launch_lr(const DmmArgs& a, cudaStream_t s)
{
    const int chains = a.which == 0 ? a.H : a.W;
    if (a.L == 32 * LPT)
        dmm_pass_kernel<LPT, R, false><<<chains, kWarps * 32, 0, s>>>(a);
    else
        dmm_pass_kernel<LPT, R, true><<<chains, kWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

template <int LPT>
cudaError_t launch_l(const DmmArgs& a, int radius, cudaStream_t s)
{
    switch (radius) {
        case 1: return launch_lr<LPT, 1>(a, s);
        case 2: return launch_lr<LPT, 2>(a, s);
        case 3: return launch_lr<LPT, 3>(a, s);
        default: return launch_lr<LPT, 4>(a, s);
    }
}

}  // namespace

cudaError_t launch_dmm_pass(const DmmArgs& a, int lpt, int radius, cudaStream_t s)
{
    switch (lpt) {
        case 1: return launch_l<1>(a, radius, s);
        case 2: return launch_l<2>(a, radius, s);
        case 4: return launch_l<4>(a, radius, s);
        default: return launch_l<8>(a, radius, s);
    }
}

}  // namespace dm
