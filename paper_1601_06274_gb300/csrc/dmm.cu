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
// unaries, stored message and mu are loaded one step ahead (dmm_alt_kernel,
// any L); for L a multiple of 16, dmm_alt_staged_kernel below copies them
// NS - 1 steps ahead into shared memory.
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

// ---------------------------------------------------------------------------
// Staged form of the alternative minorants (label counts that are multiples of
// 16).  Same chain, same arithmetic and the same results as dmm_alt_kernel,
// bit for bit; what changes is how a node's inputs reach the warp.  A chain has
// one warp and its steps depend on one another, so a load issued one step ahead
// leaves most of a DRAM round trip exposed at every step.  Here every input of
// a node -- its lambda_in row, its cost row, the stored message of the other
// direction, its mu (lambda_out of the previous pass) and the word holding the
// weight of the edge the sweep leaves it by -- is copied into a ring of NS node
// slots in shared memory by cp.async, NS - 1 steps ahead, one commit group per
// step.  Copies are 16 bytes where the rows allow it: lambda rows of LPT int32
// per lane (L a multiple of LPT, so every chunk is aligned and whole), cost
// rows of L or 2L bytes in 16-byte chunks (L a multiple of 16).  The edge
// weight comes with its aligned 4-byte word (the workspace's weight arrays
// start on 256-byte boundaries, so the word stays inside its array).
// A step is also cut down to what the chain needs: the node's pixel advances
// by a constant stride per sweep (32-bit element offsets), a lane's labels are
// all in or all out (one test per lane, not per label), the form of the
// rounding floor(gamma m) is chosen once per sweep, and the penalty taps come
// from a copy of the table in shared memory.  Measured on the 1242x375x128
// frame with the iterative minorant: a horizontal pass 6.04 -> 1.90 ms (375
// warps; latency-bound), a vertical pass 1.66 -> 0.72 ms (1242 warps; DRAM at
// two thirds of its peak: the int32 messages and mu of four sweeps per chain).
// ---------------------------------------------------------------------------

// BYTES of read-only data of the pass (16-byte pieces bypass L1), or with OWN
// data this warp wrote earlier in the launch (through L1, which holds the
// SM's own writes)
template <int BYTES, bool OWN = false>
__device__ __forceinline__ void cp_async_n(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 32) {
        cp_async_n<16, OWN>(smem, gmem);
        cp_async_n<16, OWN>(static_cast<char*>(smem) + 16, static_cast<const char*>(gmem) + 16);
    } else if constexpr (BYTES == 16 && !OWN) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES)
                     : "memory");
    }
}
__device__ __forceinline__ void cp_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// one node slot of the ring: lambda_in row, mu row, other-direction message,
// cost row (room for uint16), edge-weight word
template <int LPT>
struct AltSlot {
    static constexpr int KP = 32 * LPT;
    static constexpr int LAM = 0, MU = 4 * KP, OTH = 8 * KP, COST = 12 * KP, WORD = 14 * KP;
    static constexpr int BYTES = 14 * KP + 16;
};

template <int LPT>
constexpr int alt_ring_slots() { return 8; }

template <int LPT>
constexpr int alt_ring_bytes() { return alt_ring_slots<LPT>() * AltSlot<LPT>::BYTES; }

// One sweep of the staged kernel, fixed for its steps: node k0 + dir t at step
// t, its pixel P0 + DP t (DP = dir times the pixel stride of the chain), the
// edge it leaves by at pixel offset EOFF from it (every step but the last of a
// pass has one; the initial backward sweep stops one node short, so all of its
// steps do).  Element offsets stay below H W L < 2^31 (dm_create's bound).
struct AltSweep {
    const int32_t* obuf;  // stored messages of the other direction (nullptr: none)
    int k0, dir, P0, DP, EOFF, nedge;  // steps t < nedge have an edge
    bool with_mu;
};

// cp.async every input of step t's node into slot `slot`
template <int LPT, bool PAD>
__device__ __forceinline__ void alt_issue(const DmmArgs& A, const Chain& ch, const AltSweep& sw, int t,
                                          unsigned char* slot, int lane, bool lane_in, int cost_chunks)
{
    using S = AltSlot<LPT>;
    const int p = sw.P0 + sw.DP * t;
    const int eo = p * ch.L + lane * LPT;
    if (!PAD || lane_in) {
        cp_async_n<4 * LPT>(slot + S::LAM + lane * 4 * LPT, A.lam_in + eo);
        if (sw.with_mu) cp_async_n<4 * LPT, true>(slot + S::MU + lane * 4 * LPT, A.lam_out + eo);
    }
    if (sw.obuf != nullptr)
        cp_async_n<4 * LPT, true>(slot + S::OTH + lane * 4 * LPT,
                                  sw.obuf + (sw.k0 + sw.dir * t) * (32 * LPT) + lane * LPT);
    if (lane < cost_chunks) {  // 16-byte chunks of the cost row (rows only)
        const unsigned char* row = A.cost16 != nullptr
                                       ? reinterpret_cast<const unsigned char*>(A.cost16 + p * ch.L)
                                       : A.cost + p * ch.L;
        cp_async_n<16>(slot + S::COST + lane * 16, row + lane * 16);
    }
    if (lane == 0 && t < sw.nedge) cp_async_n<4>(slot + S::WORD, A.wedge + ((p + sw.EOFF) & ~3));
}

// step t's node inputs from its slot: theta = lambda_in (+ cost on rows),
// padding labels infinite; mu 0 when not staged or past L; the weight (or -1)
template <int LPT, bool PAD>
__device__ __forceinline__ void alt_read(const DmmArgs& A, const Chain& ch, const AltSweep& sw, int t,
                                         const unsigned char* slot, int lane, bool lane_in, int (&lam)[LPT],
                                         NodeIn<LPT>& nd)
{
    using S = AltSlot<LPT>;
    const int* sl = reinterpret_cast<const int*>(slot + S::LAM) + lane * LPT;
    const int* sm = reinterpret_cast<const int*>(slot + S::MU) + lane * LPT;
    const int* so = reinterpret_cast<const int*>(slot + S::OTH) + lane * LPT;
    const bool in = !PAD || lane_in;  // L is a multiple of LPT: a lane's labels are all in or all out
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        lam[j] = in ? sl[j] : 0;
        nd.mu[j] = (sw.with_mu && in) ? sm[j] : 0;
        nd.other[j] = sw.obuf != nullptr ? so[j] : 0;
    }
    if (ch.which == 0) {
        if (A.cost16 != nullptr) {
            const uint16_t* c = reinterpret_cast<const uint16_t*>(slot + S::COST) + lane * LPT;
#pragma unroll
            for (int j = 0; j < LPT; ++j) nd.th[j] = in ? lam[j] + (int)c[j] : kInf;
        } else {
            const unsigned char* c = slot + S::COST + lane * LPT;
#pragma unroll
            for (int j = 0; j < LPT; ++j) nd.th[j] = in ? lam[j] + (int)c[j] : kInf;
        }
    } else {
#pragma unroll
        for (int j = 0; j < LPT; ++j) nd.th[j] = in ? lam[j] : kInf;
    }
    if (t < sw.nedge) {
        const int pe = sw.P0 + sw.DP * t + sw.EOFF;
        nd.om = (int)((*reinterpret_cast<const uint32_t*>(slot + S::WORD) >> (8 * (pe & 3))) & 0xffu);
    } else {
        nd.om = -1;
    }
}

// the last visit of a node with lambda_in taken from its slot: what
// finalise_node does
template <int LPT, bool PAD>
__device__ __forceinline__ void alt_finalise(const DmmArgs& A, int pix, int lane, bool lane_in,
                                             const int (&mu)[LPT], const int (&lam)[LPT], long long& lb_acc)
{
    int best = kInf, arg = 0x7fffffff;
    if (!PAD || lane_in) {
        int32_t* out = A.lam_out + pix * A.L + lane * LPT;
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            out[j] = mu[j] - lam[j];
            if (mu[j] < best) {
                best = mu[j];
                arg = lane * LPT + j;
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

// penalty taps of weight om from the CTA's copy of the table (flags a weight
// without an integer table, as taps_for does)
__device__ __forceinline__ const int* taps_smem(const DmmArgs& A, const int* s_taps, int om)
{
    const int* tap = s_taps + om * kTapW;
    if (tap[kTapValid] == 0) atomicOr(A.err, kDevErrBadOmega);
    return tap;
}

template <int LPT, int R, bool PAD, int KIND>
__global__ void __launch_bounds__(32) dmm_alt_staged_kernel(const DmmArgs A)
{
    constexpr int NS = alt_ring_slots<LPT>();
    constexpr int KP = 32 * LPT;
    using S = AltSlot<LPT>;
    extern __shared__ __align__(16) unsigned char s_ring[];
    // the taps table in shared memory (a lookup per step in global memory
    // misses L1 once the streamed rows have evicted the table)
    __shared__ __align__(16) int s_taps[256 * kTapW];
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < 256 * kTapW / 4; i += 32)
        reinterpret_cast<int4*>(s_taps)[i] = __ldg(reinterpret_cast<const int4*>(A.taps) + i);
    __syncwarp();
    Chain ch;
    ch.which = A.which;
    ch.W = A.W;
    ch.L = A.L;
    ch.KP = A.KP;
    ch.n = A.which == 0 ? A.W : A.H;
    ch.c = blockIdx.x;
    const int n = ch.n;
    const int pst = A.which == 0 ? 1 : A.W;           // pixels between chain nodes
    const int pix0 = A.which == 0 ? ch.c * A.W : ch.c;  // pixel of node 0
    const bool lane_in = lane * LPT < A.L;
    const int cost_chunks = A.which == 0 ? A.L * (A.cost16 != nullptr ? 2 : 1) / 16 : 0;
    int32_t* F = A.fmsg + (size_t)ch.c * n * KP;
    int32_t* B = A.bmsg + (size_t)ch.c * n * KP;
    const int passes = KIND == 1 ? 1 : A.max_pass;
    int msgv[LPT], x[LPT], lam[LPT];
    long long lb_acc = 0;

    // A sweep of cnt steps; step(t, cur) consumes step t's node inputs.  Before
    // step t the commit groups of steps 0 .. t are complete (NS - 1 + t groups
    // committed, at most NS - 2 pending); step t + NS - 1 then goes into the
    // slot of step t - 1, which every lane has read (the __syncwarp after the
    // wait).
    auto run = [&](const AltSweep& sw, int cnt, auto step) {
#pragma unroll 1
        for (int t = 0; t < NS - 1; ++t) {
            if (t < cnt) alt_issue<LPT, PAD>(A, ch, sw, t, s_ring + t * S::BYTES, lane, lane_in, cost_chunks);
            cp_commit_group();
        }
        unsigned char* rd = s_ring;                       // slot of step t
        unsigned char* wr = s_ring + (NS - 1) * S::BYTES;  // slot of step t + NS - 1
#pragma unroll 1
        for (int t = 0; t < cnt; ++t) {
            cp_wait_group<NS - 2>();
            __syncwarp();
            NodeIn<LPT> cur;
            alt_read<LPT, PAD>(A, ch, sw, t, rd, lane, lane_in, lam, cur);
            if (t + NS - 1 < cnt) alt_issue<LPT, PAD>(A, ch, sw, t + NS - 1, wr, lane, lane_in, cost_chunks);
            cp_commit_group();
            rd = rd + S::BYTES == s_ring + NS * S::BYTES ? s_ring : rd + S::BYTES;
            wr = wr + S::BYTES == s_ring + NS * S::BYTES ? s_ring : wr + S::BYTES;
            step(t, cur);
        }
        cp_wait_group<0>();
        __syncwarp();
    };

    // backward sweep of the chain with mu = 0: B_{k-1} = Msg(theta_k + B_k),
    // k = n - 1 .. 1, over the edge (k - 1, k)
#pragma unroll
    for (int j = 0; j < LPT; ++j) msgv[j] = 0;
    store_msg<LPT>(B + (size_t)(n - 1) * KP, lane, msgv);
    {
        const AltSweep sw{nullptr, n - 1, -1, pix0 + (n - 1) * pst, -pst, -pst, n - 1, false};
        int32_t* bk = B + (size_t)(n >= 2 ? n - 2 : 0) * KP;  // the message into node k - 1
        run(sw, n - 1, [&](int t, NodeIn<LPT>& cur) {
            const int* tap = taps_smem(A, s_taps, cur.om);
#pragma unroll
            for (int j = 0; j < LPT; ++j) x[j] = cur.th[j] + msgv[j];
            msg<LPT, R, PAD>(x, msgv, tap, lane, A.L);
            store_msg<LPT>(bk, lane, msgv);
            bk -= KP;
        });
    }

#pragma unroll 1
    for (int s = 1; s <= passes; ++s) {
        const bool last = s == passes;
        const bool fwd = (s & 1) == 1;
        const int num = KIND == 1 ? 1 : (last ? 1 : A.gamma_num);
        const int den = KIND == 1 ? n : (last ? 1 : A.gamma_den);
        const int shift = (den & (den - 1)) == 0 ? __ffs(den) - 1 : -1;  // den = 2^shift
        // the form of floor(m gamma) for the whole sweep: m, m >> shift, 32-bit
        // or 64-bit division (gamma_part's cases, decided once)
        const int gform = num == den ? 0 : (num == 1 ? (shift >= 0 ? 1 : 2) : 3);
        const AltSweep sw{fwd ? B : F, fwd ? 0 : n - 1, fwd ? 1 : -1,
                          pix0 + (fwd ? 0 : (n - 1) * pst), fwd ? pst : -pst, fwd ? 0 : -pst, n - 1,
                          s > 1};
        int32_t* sk = (fwd ? F : B) + (size_t)(fwd ? 0 : n - 1) * KP;  // messages this pass forms
        const int dk = fwd ? KP : -KP;
#pragma unroll
        for (int j = 0; j < LPT; ++j) msgv[j] = 0;
        run(sw, n, [&](int t, NodeIn<LPT>& cur) {
            const int pix = sw.P0 + sw.DP * t;
            const int* tap = cur.om >= 0 ? taps_smem(A, s_taps, cur.om) : nullptr;
            if (!last) store_msg<LPT>(sk, lane, msgv);
            sk += dk;
            int m[LPT];
#pragma unroll
            for (int j = 0; j < LPT; ++j) m[j] = msgv[j] + cur.th[j] - cur.mu[j] + cur.other[j];
            if (!PAD || lane_in) {
                if (gform == 0) {
#pragma unroll
                    for (int j = 0; j < LPT; ++j) cur.mu[j] += m[j];
                } else if (gform == 1) {
#pragma unroll
                    for (int j = 0; j < LPT; ++j) cur.mu[j] += m[j] >> shift;
                } else if (gform == 2) {
#pragma unroll
                    for (int j = 0; j < LPT; ++j) cur.mu[j] += floor_div32(m[j], den);
                } else {
#pragma unroll
                    for (int j = 0; j < LPT; ++j) cur.mu[j] += floor_div64((long long)m[j] * num, den);
                }
            }
            if (last) {
                alt_finalise<LPT, PAD>(A, pix, lane, lane_in, cur.mu, lam, lb_acc);
            } else if (!PAD || lane_in) {
                int32_t* out = A.lam_out + pix * A.L + lane * LPT;
#pragma unroll
                for (int j = 0; j < LPT; ++j) out[j] = cur.mu[j];
            }
            if (t + 1 < n) {
                // the naive minorant takes the min-marginals of f itself; the
                // iterative one those of the remainder f - mu, mu_k just updated
#pragma unroll
                for (int j = 0; j < LPT; ++j)
                    x[j] = cur.th[j] - (KIND == 1 ? 0 : cur.mu[j]) + msgv[j];
                msg<LPT, R, PAD>(x, msgv, tap, lane, A.L);
            }
        });
    }
    if (A.lb != nullptr && lane == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(A.lb), (unsigned long long)lb_acc);
}

template <int LPT, int R, int KIND>
void launch_alt(const DmmArgs& a, int chains, cudaStream_t s)
{
    // label counts that are multiples of 16 (every chunk of a row whole and
    // aligned) take the staged kernel; the rest the one-step-ahead loads
    if (a.L % 16 == 0) {
        if (a.L == 32 * LPT)
            dmm_alt_staged_kernel<LPT, R, false, KIND><<<chains, 32, alt_ring_bytes<LPT>(), s>>>(a);
        else
            dmm_alt_staged_kernel<LPT, R, true, KIND><<<chains, 32, alt_ring_bytes<LPT>(), s>>>(a);
    } else if (a.L == 32 * LPT) {
        dmm_alt_kernel<LPT, R, false, KIND><<<chains, 32, 0, s>>>(a);
    } else {
        dmm_alt_kernel<LPT, R, true, KIND><<<chains, 32, 0, s>>>(a);
    }
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
