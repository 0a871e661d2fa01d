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

// ---------------------------------------------------------------------------
// Other chain minorants (Sec. 2.3 "Good and Fast Minorants"; App. A).
//   naive (KIND 1): every node takes floor(m_i / n) of its min-marginal m_i.
//   iterative (KIND 2, Alg. iterative-minorant): mu := 0, then max_pass passes
//     alternating in direction (forward first); at node i the min-marginal of
//     the remainder f - mu is F_i + theta_i - mu_i + B_i, where the message from
//     the side visited earlier in the pass is formed as the pass goes and the
//     other one was stored by the previous pass (an initial backward sweep
//     before the first), and mu_i += floor(gamma m_i), gamma = 1 on the last
//     pass.
// One warp per chain, labels across its lanes as in dmm_pass_kernel; a sweep
// stores the messages it forms (F or B) for the next pass, which runs the
// other way.  mu accumulates in lam_out; each node's final visit writes
// lam_out = mu - lam_in and takes the labels and the bound.  The next node's
// unaries, stored message and mu are loaded one step ahead.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int floor_div64(long long a, int d)
{
    return (int)(a >= 0 ? a / d : -((-a + d - 1) / d));
}

__device__ __forceinline__ int floor_div32(int a, int d)
{
    return a >= 0 ? a / d : -((-a + d - 1) / d);
}

// floor(m * num / den) for the pass's gamma = num / den (0 <= num <= den): m
// itself for gamma = 1, an arithmetic shift (a floor) for 1 / 2^s, 32-bit
// division for 1 / den, 64-bit otherwise; the case is the same for the warp
__device__ __forceinline__ int gamma_part(int m, int num, int den, int shift)
{
    if (num == den) return m;
    if (num == 1) return shift >= 0 ? (m >> shift) : floor_div32(m, den);
    return floor_div64((long long)m * num, den);
}

template <int LPT>
struct NodeIn {
    int th[LPT], other[LPT], mu[LPT];
    int om;  // weight of the edge the sweep leaves node k by (-1: none)
};

// penalty taps of weight om (flags a weight without an integer table)
__device__ __forceinline__ const int* taps_for(const DmmArgs& A, int om)
{
    const int* tap = A.taps + om * kTapW;
    if (__ldg(tap + kTapValid) == 0) atomicOr(A.err, kDevErrBadOmega);
    return tap;
}

template <int LPT>
__device__ __forceinline__ void load_node(const DmmArgs& A, const Chain& ch, const int32_t* obuf,
                                          int k, int edge, bool load_mu, int lane, NodeIn<LPT>& nd)
{
    nd.om = edge >= 0 ? (int)__ldg(A.wedge + ch.pix(edge)) : -1;
    load_theta<LPT>(A, ch, k, lane, nd.th);
    if (obuf != nullptr) load_msg<LPT>(obuf + (size_t)k * A.KP, lane, nd.other);
    const size_t base = ch.pix(k) * (size_t)ch.L + (size_t)lane * LPT;
#pragma unroll
    for (int j = 0; j < LPT; ++j)
        nd.mu[j] = (load_mu && lane * LPT + j < ch.L) ? A.lam_out[base + j] : 0;
}

// bring node k's inputs towards L2 ahead of the one-step register prefetch
// (a chain has one warp, so the latency of DRAM is not hidden by other warps)
constexpr int kL2Ahead = 8;

__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int LPT>
__device__ __forceinline__ void prefetch_node(const DmmArgs& A, const Chain& ch, const int32_t* obuf,
                                              int k, bool mu, int lane)
{
    const size_t base = ch.pix(k) * (size_t)ch.L + (size_t)lane * LPT;
    if (lane * LPT < ch.L) {
        prefetch_l2(A.lam_in + base);
        if (ch.which == 0)
            prefetch_l2(A.cost16 != nullptr ? (const void*)(A.cost16 + base)
                                            : (const void*)(A.cost + base));
        if (mu) prefetch_l2(A.lam_out + base);
    }
    if (obuf != nullptr) prefetch_l2(obuf + (size_t)k * A.KP + (size_t)lane * LPT);
}

template <int LPT>
__device__ __forceinline__ void finalise_node(const DmmArgs& A, const Chain& ch, int k, int lane,
                                              const int (&mu)[LPT], long long& lb_acc)
{
    const size_t pix = ch.pix(k);
    const size_t base = pix * (size_t)A.L + (size_t)lane * LPT;
    int best = kInf, arg = 0x7fffffff;
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int l = lane * LPT + j;
        if (l < A.L) {
            A.lam_out[base + j] = mu[j] - __ldg(A.lam_in + base + j);
            if (mu[j] < best) {            // lambda_h + lambda_v = mu
                best = mu[j];
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

template <int LPT, int R, bool PAD, int KIND>
__global__ void __launch_bounds__(32) dmm_alt_kernel(const DmmArgs A)
{
    const int lane = threadIdx.x & 31;
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
    const int passes = KIND == 1 ? 1 : A.max_pass;
    int msgv[LPT], x[LPT];
    long long lb_acc = 0;

    // backward sweep of the chain with mu = 0: B_{k-1} = Msg(theta_k + B_k)
#pragma unroll
    for (int j = 0; j < LPT; ++j) msgv[j] = 0;
    store_msg<LPT>(B + (size_t)(n - 1) * A.KP, lane, msgv);
    {
        NodeIn<LPT> cur, nxt;
        if (n > 1) load_node<LPT>(A, ch, nullptr, n - 1, n - 2, false, lane, cur);
        for (int k = n - 1; k > 0; --k) {
            if (k - kL2Ahead >= 0) prefetch_node<LPT>(A, ch, nullptr, k - kL2Ahead, false, lane);
            if (k > 1) load_node<LPT>(A, ch, nullptr, k - 1, k - 2, false, lane, nxt);
            const int* tap = taps_for(A, cur.om);
#pragma unroll
            for (int j = 0; j < LPT; ++j) x[j] = cur.th[j] + msgv[j];
            msg<LPT, R, PAD>(x, msgv, tap, lane, A.L);
            store_msg<LPT>(B + (size_t)(k - 1) * A.KP, lane, msgv);
            cur = nxt;
        }
    }

    for (int s = 1; s <= passes; ++s) {
        const bool last = s == passes;
        const bool fwd = (s & 1) == 1;
        const int num = KIND == 1 ? 1 : (last ? 1 : A.gamma_num);
        const int den = KIND == 1 ? n : (last ? 1 : A.gamma_den);
        const int shift = (den & (den - 1)) == 0 ? __ffs(den) - 1 : -1;  // den = 2^shift
        int32_t* obuf = fwd ? B : F;     // messages from the side not yet visited
        int32_t* sbuf = fwd ? F : B;     // messages this pass forms, kept for the next
#pragma unroll
        for (int j = 0; j < LPT; ++j) msgv[j] = 0;
        NodeIn<LPT> cur, nxt;
        // node k's outgoing edge: k (forward) or k - 1 (backward), none at the far end
        auto edge_of = [&](int k) { return fwd ? (k + 1 < n ? k : -1) : k - 1; };
        load_node<LPT>(A, ch, obuf, fwd ? 0 : n - 1, edge_of(fwd ? 0 : n - 1), s > 1, lane, cur);
        for (int t = 0; t < n; ++t) {
            const int k = fwd ? t : n - 1 - t;
            if (t + kL2Ahead < n)
                prefetch_node<LPT>(A, ch, obuf, fwd ? k + kL2Ahead : k - kL2Ahead, s > 1, lane);
            if (t + 1 < n)
                load_node<LPT>(A, ch, obuf, fwd ? k + 1 : k - 1, edge_of(fwd ? k + 1 : k - 1),
                               s > 1, lane, nxt);
            const int* tap = cur.om >= 0 ? taps_for(A, cur.om) : nullptr;
            if (!last) store_msg<LPT>(sbuf + (size_t)k * A.KP, lane, msgv);
#pragma unroll
            for (int j = 0; j < LPT; ++j) {
                if (lane * LPT + j < A.L) {
                    const int m = msgv[j] + cur.th[j] - cur.mu[j] + cur.other[j];
                    cur.mu[j] += gamma_part(m, num, den, shift);
                }
            }
            if (last) {
                finalise_node<LPT>(A, ch, k, lane, cur.mu, lb_acc);
            } else {
                const size_t base = ch.pix(k) * (size_t)ch.L + (size_t)lane * LPT;
#pragma unroll
                for (int j = 0; j < LPT; ++j)
                    if (lane * LPT + j < A.L) A.lam_out[base + j] = cur.mu[j];
            }
            if (t + 1 < n) {
                // the naive minorant takes the min-marginals of f itself; the
                // iterative one those of the remainder f - mu, mu_k just updated
#pragma unroll
                for (int j = 0; j < LPT; ++j)
                    x[j] = cur.th[j] - (KIND == 1 ? 0 : cur.mu[j]) + msgv[j];
                msg<LPT, R, PAD>(x, msgv, tap, lane, A.L);
                cur = nxt;
            }
        }
    }
    if (A.lb != nullptr && lane == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(A.lb), (unsigned long long)lb_acc);
}

template <int LPT, int R, int KIND>
void launch_alt(const DmmArgs& a, int chains, cudaStream_t s)
{
    if (a.L == 32 * LPT)
        dmm_alt_kernel<LPT, R, false, KIND><<<chains, 32, 0, s>>>(a);
    else
        dmm_alt_kernel<LPT, R, true, KIND><<<chains, 32, 0, s>>>(a);
}

template <int LPT, int R>
cudaError_t launch_lr(const DmmArgs& a, cudaStream_t s)
{
    const int chains = a.which == 0 ? a.H : a.W;
    if (a.minorant == 1)
        launch_alt<LPT, R, 1>(a, chains, s);
    else if (a.minorant == 2)
        launch_alt<LPT, R, 2>(a, chains, s);
    else if (a.L == 32 * LPT)
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
