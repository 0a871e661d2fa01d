// Dual MM pass with packed 16-bit message arithmetic (the fast path): device
// code, kernels and launchers, included by one translation unit per label
// class (dmm16_np*_*.cu) so that the classes compile in parallel.
//
// Same algorithm as dmm.cu -- Alg. Dual_MM of arXiv 1601.06274 with the
// hierarchical minorant of App. A (Alg. Handshake) -- and bit-identical
// results, organised for throughput:
//
// * Values.  Every message is stored as an int16 vector plus an int32 scalar
//   offset.  After each Msg the vector is shifted by an even number so that
//   its minimum is 0 or 1; a message's range is at most omega*C (its values lie
//   in [min a, min a + omega C]), so vectors stay tiny.  Even shifts commute with
//   the Handshake's floor(m/2): floor((v + 2k)/2) = floor(v/2) + k.  Duals are
//   stored the same way: an int32 base per pixel plus a vector of deltas
//   (uint8 or int16).  With the horizontal pass writing lambda_h = c + Lin +
//   Rin and the vertical pass lambda_v = Lin + Rin, the deltas are bounded by
//   max(c) + 2(omega C + 1), which the host checks before choosing this path.
// * Arithmetic.  Two adjacent labels share one 32-bit register; vadd2/vmins2
//   and the DPX add-min (viaddmin_s16x2) process both at once.  Each lane
//   holds 2*NP consecutive labels.
// * Messages.  Msg(a)(x') = min(a(x'), min_{d<=R}(min a(x'-d), a(x'+d)) + T_d,
//   min(a) + P2): shuffles bring the R neighbouring labels from the adjacent
//   lanes, one redux.sync gives min(a).
// * Memory.  The unaries of the next PF sweep steps are prefetched into a
//   register ring.  A sweep stores only the messages a later level reads (the
//   split points along the spine of the sub-chain it leaves behind); a
//   Handshake writes the boundary messages of its children, or, for a child
//   that is a single node, that node's output directly.
// * Schedule.  One CTA (8 warps) per chain.  Level 0: two warps sweep the two
//   halves, one warp does the Handshake.  Level l >= 1: one warp per segment
//   does its sweep and its Handshake; __syncthreads between levels.

#pragma once

#include <atomic>

#include "dm_internal.cuh"

namespace dm {
namespace k16 {

constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kInf2 = 0x3FFF3FFFu;  // 16383 in both halves: never the minimum

__device__ __forceinline__ uint32_t vadd2(uint32_t a, uint32_t b) { return __vadd2(a, b); }
__device__ __forceinline__ uint32_t vsub2(uint32_t a, uint32_t b) { return __vsub2(a, b); }
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) { return __vmins2(a, b); }
__device__ __forceinline__ uint32_t addmin2(uint32_t a, uint32_t b, uint32_t c)
{
    return __viaddmin_s16x2(a, b, c);  // min(a + b, c) per 16-bit half
}
__device__ __forceinline__ uint32_t splat(int v) { return ((uint32_t)v & 0xffffu) * 0x10001u; }
__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t v) { return (int)v >> 16; }

struct Taps {
    uint32_t t[kRMax];  // T_d in both halves
    int p2;
};

// value (packed pair) of this lane's register index IDX (may be outside [0, NP))
template <int NP, int IDX>
__device__ __forceinline__ uint32_t ext_reg(const uint32_t (&a)[NP], int lane)
{
    constexpr int off = (IDX >= 0) ? IDX / NP : -((-IDX + NP - 1) / NP);  // floor(IDX / NP)
    constexpr int loc = IDX - off * NP;
    if constexpr (off == 0) {
        return a[loc];
    } else if constexpr (off < 0) {
        const uint32_t v = __shfl_up_sync(kFull, a[loc], -off);
        return (lane + off >= 0) ? v : kInf2;
    } else {
        const uint32_t v = __shfl_down_sync(kFull, a[loc], off);
        return (lane + off <= 31) ? v : kInf2;
    }
}

template <int NP, int H, int IDX>
__device__ __forceinline__ void fill_ext(const uint32_t (&a)[NP], uint32_t (&E)[NP + 2 * H],
                                         int lane)
{
    if constexpr (IDX < NP + H) {
        E[IDX + H] = ext_reg<NP, IDX>(a, lane);
        fill_ext<NP, H, IDX + 1>(a, E, lane);
    }
}

// out = Msg(a) normalised, with the scalar offset `off` of `a` turned into
// that of out.  `pad` marks a lane whose labels are all >= L.
template <int NP, int R, bool PAD>
__device__ __forceinline__ void msg16(uint32_t (&a)[NP], uint32_t (&out)[NP], int& off,
                                      const Taps& tp, int lane, bool pad)
{
    constexpr int H = (R + 1) / 2;
    if constexpr (PAD) {
#pragma unroll
        for (int p = 0; p < NP; ++p) a[p] = pad ? kInf2 : a[p];
    }
    uint32_t mm = a[0];
#pragma unroll
    for (int p = 1; p < NP; ++p) mm = vmin2(mm, a[p]);
    const int m = __reduce_min_sync(kFull, min(lo16(mm), hi16(mm)));
    uint32_t E[NP + 2 * H];
    fill_ext<NP, H, -H>(a, E, lane);
    const int shift = m & ~1;                       // even floor of the minimum
    const uint32_t negs = splat(-shift);
    const uint32_t caps = splat(m - shift + tp.p2); // (min a + P2) - shift
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint32_t res = a[p];
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            uint32_t l, r;
            if (d & 1) {  // labels (2p-d, 2p+1-d) and (2p+d, 2p+1+d) straddle two registers
                l = __byte_perm(E[p - (d + 1) / 2 + H], E[p - (d - 1) / 2 + H], 0x5432);
                r = __byte_perm(E[p + (d - 1) / 2 + H], E[p + (d + 1) / 2 + H], 0x5432);
            } else {
                l = E[p - d / 2 + H];
                r = E[p + d / 2 + H];
            }
            res = addmin2(vmin2(l, r), tp.t[d - 1], res);
        }
        out[p] = addmin2(res, negs, caps);  // min(res, min a + P2) - shift
    }
    off += shift;
}

struct Ctx16 {
    int which, H, W, L, n, c, KP2;  // KP2: packed registers per stored message (32 * NP)
    bool c16;                       // uint16 cost volume
    int32_t* err;                   // the device error word
    __device__ __forceinline__ int pix(int k) const { return which == 0 ? c * W + k : k * W + c; }
};

// Checked builds (-DDM_CHECKED, the library's memory-safety test) verify every
// node, edge and message position before a global access: a position outside
// the chain sets kDevErrIndex and skips the access.  Otherwise the checks
// compile away.
#ifdef DM_CHECKED
__device__ __forceinline__ bool in_chain(const Ctx16& C, int k, int limit)
{
    const bool ok = k >= 0 && k < limit && C.c >= 0 && C.c < (C.which == 0 ? C.H : C.W);
    if (!ok) atomicOr(C.err, kDevErrIndex);
    return ok;
}
#else
__device__ __forceinline__ bool in_chain(const Ctx16&, int, int) { return true; }
#endif

// ---------------------------------------------------------------------------
// Asynchronous staging.  Unary rows and messages reach shared memory through
// cp.async; completion is tracked per commit group, so many sweep steps are in
// flight without tying up the warp's register scoreboards.
// ---------------------------------------------------------------------------

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// copy `bytes` (a multiple of 4) in units of the largest of 16, 8, 4 bytes that
// divides it; source and destination are aligned to that unit
__device__ __forceinline__ void cp_bytes(uint8_t* dst, const uint8_t* src, int bytes)
{
    if ((bytes & 15) == 0) {
        for (int o = 0; o < bytes; o += 16) cp_async<16>(dst + o, src + o);
    } else if ((bytes & 7) == 0) {
        for (int o = 0; o < bytes; o += 8) cp_async<8>(dst + o, src + o);
    } else {
        for (int o = 0; o < bytes; o += 4) cp_async<4>(dst + o, src + o);
    }
}

constexpr int kBlk = 8;  // sweep steps staged per block (two blocks in flight)
constexpr int kL0 = 3;   // levels below this one are walked per warp without barriers

// shared-memory geometry
template <int NP, typename DT>
struct Geo {
    static constexpr int ROW = 64 * NP * (int)sizeof(DT);  // unary row of 64 NP labels
    static constexpr int CROW = 128 * NP;                   // cost row (uint8 or uint16)
    static constexpr int BLK = kBlk * ROW + 64;             // rows, 8 bases, 8 omega words
    static constexpr int NODE = ROW + CROW + 16;            // Handshake node: row, cost, base, omega
    static constexpr int MSG = 128 * NP + 16;               // packed message + offset
    static constexpr int WARP = 2 * BLK + 4 * NODE + 2 * MSG;
};

// Stage the unaries of sweep steps u = 0..cnt-1 (nodes k0 + dir*u) into a block:
// four lanes per row, lanes 0-7 the bases, lanes 8-15 the words holding the
// weights of the edges the steps use.
template <int NP, typename DT>
__device__ __forceinline__ void issue_block(const Dmm16Args& A, const Ctx16& C, int k0, int dir,
                                            int cnt, uint8_t* blk, int lane)
{
    using G = Geo<NP, DT>;
    const int rowd = C.L * (int)sizeof(DT);
    const int part = rowd >> 2;
    const int u = lane >> 2, q = lane & 3;
    if (u < cnt && in_chain(C, k0 + dir * u, C.n)) {
        const int pix = C.pix(k0 + dir * u);
        cp_bytes(blk + u * G::ROW + q * part,
                 reinterpret_cast<const uint8_t*>(A.delta_in) + (size_t)pix * rowd + q * part, part);
    }
    if (lane < cnt && in_chain(C, k0 + dir * lane, C.n))
        cp_async<4>(blk + kBlk * G::ROW + 4 * lane, A.base_in + C.pix(k0 + dir * lane));
    const int v = lane - 8;
    if (v >= 0 && v < cnt) {
        const int k = k0 + dir * v;
        const int e = dir > 0 ? k : k - 1;  // the edge (e, e + 1) the step crosses
        if (in_chain(C, e, C.n - 1))
            cp_async<4>(blk + kBlk * G::ROW + 32 + 4 * v, A.wedge + (C.pix(e) & ~3));
    }
}

// stage node k (row, cost row, base, weight of edge `edge` or none) for a Handshake
template <int NP, typename DT>
__device__ __forceinline__ void issue_node(const Dmm16Args& A, const Ctx16& C, int k, int edge,
                                           uint8_t* slot, int lane)
{
    using G = Geo<NP, DT>;
    if (!in_chain(C, k, C.n) || (edge >= 0 && !in_chain(C, edge, C.n - 1))) return;
    const int pix = C.pix(k);
    const int rowd = C.L * (int)sizeof(DT);
    const int part = rowd >> 2;
    const int q = lane & 3;
    if (lane < 4)
        cp_bytes(slot + q * part, reinterpret_cast<const uint8_t*>(A.delta_in) + (size_t)pix * rowd + q * part,
                 part);
    else if (lane < 8) {
        if (A.cost16 != nullptr)
            cp_bytes(slot + G::ROW + q * (C.L >> 1),
                     reinterpret_cast<const uint8_t*>(A.cost16 + (size_t)pix * C.L) + q * (C.L >> 1),
                     C.L >> 1);
        else
            cp_bytes(slot + G::ROW + q * (C.L >> 2), A.cost + (size_t)pix * C.L + q * (C.L >> 2),
                     C.L >> 2);
    }
    else if (lane == 8)
        cp_async<4>(slot + G::ROW + G::CROW, A.base_in + pix);
    else if (lane == 9 && edge >= 0)
        cp_async<4>(slot + G::ROW + G::CROW + 4, A.wedge + (C.pix(edge) & ~3));
}

// stage message `pos` of buffer (buf, ofs) into a message slot
template <int NP>
__device__ __forceinline__ void issue_msg(const uint32_t* buf, const int* ofs, const Ctx16& C,
                                          int pos, uint8_t* slot, int lane)
{
    if (!in_chain(C, pos, C.n)) return;
    const int node = C.c * C.n + pos;
    cp_async<4 * NP>(slot + lane * 4 * NP, buf + (size_t)node * C.KP2 + lane * NP);
    if (lane == 0) cp_async<4>(slot + 128 * NP, ofs + node);
}

template <int NP>
__device__ __forceinline__ void read_msg(const uint8_t* slot, int lane, uint32_t (&m)[NP], int& off)
{
    const uint32_t* p = reinterpret_cast<const uint32_t*>(slot) + lane * NP;
#pragma unroll
    for (int q = 0; q < NP; ++q) m[q] = p[q];
    off = *reinterpret_cast<const int*>(slot + 128 * NP);
}

// byte pair p of a little-endian byte vector -> two zero-extended 16-bit halves
__device__ __forceinline__ uint32_t unpack_pair(uint32_t word, int p)
{
    return (p & 1) ? __byte_perm(word, 0, 0x4342) : __byte_perm(word, 0, 0x4140);
}

// this lane's labels of a staged row as packed 16-bit pairs
template <int NP, typename DT>
__device__ __forceinline__ void read_row(const uint8_t* row, int lane, bool pad, uint32_t (&th)[NP])
{
    if constexpr (sizeof(DT) == 1) {
        uint32_t w[(2 * NP + 3) / 4];
        const uint8_t* p = row + lane * 2 * NP;
        if constexpr (NP == 1) w[0] = *reinterpret_cast<const uint16_t*>(p);
        else if constexpr (NP == 2) w[0] = *reinterpret_cast<const uint32_t*>(p);
        else { const uint2 v = *reinterpret_cast<const uint2*>(p); w[0] = v.x; w[1] = v.y; }
#pragma unroll
        for (int q = 0; q < NP; ++q) th[q] = pad ? kInf2 : unpack_pair(w[q >> 1], q);
    } else {
        const uint32_t* p = reinterpret_cast<const uint32_t*>(row + lane * 4 * NP);
#pragma unroll
        for (int q = 0; q < NP; ++q) th[q] = pad ? kInf2 : p[q];
    }
}

// costs of this lane's labels as packed 16-bit pairs (a staged uint8 or uint16 row)
template <int NP>
__device__ __forceinline__ void read_cost(const uint8_t* crow, int lane, bool c16, uint32_t (&cv)[NP])
{
    if (c16) {
        const uint32_t* p = reinterpret_cast<const uint32_t*>(crow + lane * 4 * NP);
#pragma unroll
        for (int q = 0; q < NP; ++q) cv[q] = p[q];
        return;
    }
    uint32_t w[(2 * NP + 3) / 4];
    const uint8_t* p = crow + lane * 2 * NP;
    if constexpr (NP == 1) w[0] = *reinterpret_cast<const uint16_t*>(p);
    else if constexpr (NP == 2) w[0] = *reinterpret_cast<const uint32_t*>(p);
    else { const uint2 v = *reinterpret_cast<const uint2*>(p); w[0] = v.x; w[1] = v.y; }
#pragma unroll
    for (int q = 0; q < NP; ++q) cv[q] = unpack_pair(w[q >> 1], q);
}

// taps row of omega: {T1, T2, P2, valid, T3, T4, -, -}, T_d in both halves
template <int R>
__device__ __forceinline__ Taps taps_of(const uint32_t* s_taps, int om)
{
    const uint4 v = *reinterpret_cast<const uint4*>(s_taps + om * kTapW);
    Taps t;
    t.t[0] = v.x;
    t.t[1] = v.y;
    t.p2 = (int)v.z;
    if constexpr (R > 2) {
        const uint2 w = *reinterpret_cast<const uint2*>(s_taps + om * kTapW + 4);
        t.t[2] = w.x;
        t.t[3] = w.y;
    } else {
        t.t[2] = t.t[3] = 0u;
    }
    return t;
}

template <int NP>
__device__ __forceinline__ void store_msg(uint32_t* buf, int* ofs, const Ctx16& C, int pos,
                                          int lane, const uint32_t (&m)[NP], int off)
{
    if (!in_chain(C, pos, C.n)) return;
    uint32_t* p = buf + (size_t)(C.c * C.n + pos) * C.KP2 + lane * NP;
    if constexpr (NP == 1) p[0] = m[0];
    else if constexpr (NP == 2) *reinterpret_cast<uint2*>(p) = make_uint2(m[0], m[1]);
    else *reinterpret_cast<uint4*>(p) = make_uint4(m[0], m[1], m[2], m[3]);
    if (lane == 0) ofs[C.c * C.n + pos] = off;
}

// Output of a node that is a single node of the hierarchy: it keeps
// theta + Lin + Rin.  The horizontal pass stores lambda_h = c + Lin + Rin.  The
// vertical pass has lambda_v = Lin + Rin and stores c + lambda_v, the unary of
// the next horizontal pass (lambda_v itself is c + lambda_v - c); it can also
// emit the label and the node's share of the lower bound, the minimum over
// labels of lambda_h + lambda_v = theta + Lin + Rin.
template <int NP, typename DT>
__device__ __forceinline__ void finalise(const Dmm16Args& A, const Ctx16& C, int k, int lane,
                                         bool pad, const uint32_t (&th)[NP], int th_base,
                                         const uint32_t (&cv)[NP], const uint32_t (&lin)[NP],
                                         int lin_off, const uint32_t (&rin)[NP], int rin_off,
                                         long long& lb_acc)
{
    if (!in_chain(C, k, C.n)) return;  // k is uniform over the warp
    const int pix = C.pix(k);
    uint32_t v[NP];
    uint32_t bad = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        v[p] = vadd2(vadd2(lin[p], rin[p]), cv[p]);
        bad |= v[p];
    }
    if (lane == 0) A.base_out[pix] = lin_off + rin_off;
    if (!pad) {
        if constexpr (sizeof(DT) == 1) {
            // every delta is in [0, 255]: the host only picks 8-bit storage when it must be
            if (bad & 0xff00ff00u) atomicOr(A.err, kDevErrRange);
            uint8_t* dp = reinterpret_cast<uint8_t*>(A.delta_out) + (size_t)pix * C.L + lane * 2 * NP;
            if constexpr (NP == 1) {
                *reinterpret_cast<uint16_t*>(dp) = (uint16_t)__byte_perm(v[0], 0, 0x4420);
            } else if constexpr (NP == 2) {
                *reinterpret_cast<uint32_t*>(dp) = __byte_perm(v[0], v[1], 0x6420);
            } else {
                *reinterpret_cast<uint2*>(dp) = make_uint2(__byte_perm(v[0], v[1], 0x6420),
                                                           __byte_perm(v[2], v[3], 0x6420));
            }
        } else {
            uint32_t* dp = reinterpret_cast<uint32_t*>(reinterpret_cast<int16_t*>(A.delta_out) +
                                                       (size_t)pix * C.L + lane * 2 * NP);
            if constexpr (NP == 1) dp[0] = v[0];
            else if constexpr (NP == 2) *reinterpret_cast<uint2*>(dp) = make_uint2(v[0], v[1]);
            else *reinterpret_cast<uint4*>(dp) = make_uint4(v[0], v[1], v[2], v[3]);
        }
    }
    if (A.labels != nullptr || A.lb != nullptr) {
        int best = 0x7fffffff, arg = 0x7fffffff;
        if (!pad) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const uint32_t nu = vadd2(vadd2(lin[p], rin[p]), th[p]);
                const int a0 = lo16(nu), a1 = hi16(nu);
                if (a0 < best) { best = a0; arg = lane * 2 * NP + 2 * p; }
                if (a1 < best) { best = a1; arg = lane * 2 * NP + 2 * p + 1; }
            }
        }
        const int m = __reduce_min_sync(kFull, best);
        if (A.labels != nullptr) {
            const int am = __reduce_min_sync(kFull, best == m ? arg : 0x7fffffff);
            if (lane == 0) A.labels[pix] = (uint16_t)am;
        }
        if (lane == 0) lb_acc += (long long)m + th_base + lin_off + rin_off;
    }
}

// Segment s of level `level` of the split tree of [0, n) (the left part of a
// split keeps ceil(len/2) nodes).  Returns false if an ancestor is a single node.
// `plen` receives the length of its parent (n for the root).
__device__ __forceinline__ bool segment16(int n, int level, int s, int& a, int& b, int& plen)
{
    a = 0;
    b = n - 1;
    plen = n;
    for (int bit = level - 1; bit >= 0; --bit) {
        const int len = b - a + 1;
        if (len == 1) return false;
        plen = len;
        const int i = a + ((len + 1) >> 1) - 1;
        if ((s >> bit) & 1) a = i + 1;
        else b = i;
    }
    return true;
}

// The messages a fresh sweep must leave behind are the ones a later segment of
// at least 5 nodes inherits (segments of 2-4 nodes recompute theirs).
// Forward sweep of a segment whose left part is [a, i] (D = i - a): the split
// point of the left part, of its left part, and so on, at a + (D >> t), needed
// while that part has at least 5 nodes, i.e. (D >> (t-1)) >= 4.  Backward sweep
// whose right part is [j, b] (E = b - j + 1): the first node of the right part
// of [j, b], of its right part, and so on, at b + 1 - (E >> t), needed while
// (E >> (t-1)) >= 5.  Both are visited with t decreasing.
struct Spine {
    int t, base, span, dir;  // position(t) = base + dir * f(span >> t)
    __device__ __forceinline__ int pos() const
    {
        return t <= 0 ? -1 : (dir > 0 ? base + (span >> t) : base + 1 - (span >> t));
    }
};

__device__ __forceinline__ Spine spine_fwd(int a, int i)
{
    Spine sp{0, a, i - a, +1};
    while ((sp.span >> sp.t) >= 4) ++sp.t;  // largest t with (D >> (t-1)) >= 4
    return sp;
}

__device__ __forceinline__ Spine spine_bwd(int j, int b)
{
    Spine sp{0, b, b - j + 1, -1};
    while ((sp.span >> sp.t) >= 5) ++sp.t;  // largest t with (E >> (t-1)) >= 5
    return sp;
}

// one Msg step of a sweep from staged block data (u: index within the block)
template <int NP, int R, bool PAD, typename DT>
__device__ __forceinline__ void sweep_step(const Ctx16& C, const uint32_t* s_taps,
                                           const uint8_t* blk, int u, int k, int dir,
                                           uint32_t (&msg)[NP], int& off, int lane, bool pad)
{
    using G = Geo<NP, DT>;
    uint32_t th[NP], x[NP];
    read_row<NP, DT>(blk + u * G::ROW, lane, pad, th);
    const int e = dir > 0 ? k : k - 1;
    const uint32_t w = *reinterpret_cast<const uint32_t*>(blk + kBlk * G::ROW + 32 + 4 * u);
    const Taps tp = taps_of<R>(s_taps, (int)((w >> (8 * (C.pix(e) & 3))) & 0xffu));
    off += *reinterpret_cast<const int*>(blk + kBlk * G::ROW + 4 * u);
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = vadd2(th[p], msg[p]);
    msg16<NP, R, PAD>(x, msg, off, tp, lane, pad);
}

// One sweep of `count` Msg steps.  dir = +1: forward from node k0 (messages
// enter k0+1, k0+2, ...; edge of step k is k).  dir = -1: backward from k0
// (messages enter k0-1, ...; edge of step k is k-1).  `msg`/`off` hold the
// boundary message on entry and the last message on exit.  Messages entering
// the spine positions of `sp` are stored.  All async copies committed before
// the call must be complete.
template <int NP, int R, bool PAD, typename DT>
__device__ __forceinline__ void sweep16(const Dmm16Args& A, const Ctx16& C, const uint32_t* s_taps,
                                        uint8_t* ring, int k0, int dir, int count,
                                        uint32_t (&msg)[NP], int& off, Spine sp,
                                        uint32_t* sbuf, int* sofs, int lane, bool pad)
{
    using G = Geo<NP, DT>;
    if (count <= 0) return;
    const int nblk = (count + kBlk - 1) / kBlk;
    issue_block<NP, DT>(A, C, k0, dir, min(count, kBlk), ring, lane);
    cp_commit();
    if (nblk > 1)
        issue_block<NP, DT>(A, C, k0 + dir * kBlk, dir, min(count - kBlk, kBlk), ring + G::BLK, lane);
    cp_commit();
    int next = sp.pos();
    for (int bi = 0; bi < nblk; ++bi) {
        cp_wait<1>();
        __syncwarp();
        uint8_t* blk = ring + (bi & 1) * G::BLK;
        const int kb = k0 + dir * kBlk * bi;
        const int cnt = min(count - kBlk * bi, kBlk);
        // one copy of the step (each step depends on the previous message, so
        // unrolling buys no overlap, only instruction-cache footprint)
#pragma unroll 1
        for (int u = 0; u < cnt; ++u) {
            const int k = kb + dir * u;
            sweep_step<NP, R, PAD, DT>(C, s_taps, blk, u, k, dir, msg, off, lane, pad);
            if (k + dir == next) {
                store_msg<NP>(sbuf, sofs, C, k + dir, lane, msg, off);
                --sp.t;
                next = sp.pos();
            }
        }
        __syncwarp();
        if (bi + 2 < nblk)
            issue_block<NP, DT>(A, C, kb + dir * 2 * kBlk, dir, min(count - kBlk * (bi + 2), kBlk),
                                blk, lane);
        cp_commit();
    }
}

// A staged node: unary vector, cost vector, base, and the weight of the edge
// that was staged with it.
template <int NP>
struct Node {
    uint32_t th[NP], cv[NP];
    int base, om;
};

template <int NP, typename DT>
__device__ __forceinline__ Node<NP> read_node(const uint8_t* slot, const Ctx16& C, int edge, int lane,
                                              bool pad)
{
    using G = Geo<NP, DT>;
    Node<NP> v;
    read_row<NP, DT>(slot, lane, pad, v.th);
    read_cost<NP>(slot + G::ROW, lane, C.c16, v.cv);
    v.base = *reinterpret_cast<const int*>(slot + G::ROW + G::CROW);
    const uint32_t w = *reinterpret_cast<const uint32_t*>(slot + G::ROW + G::CROW + 4);
    v.om = edge >= 0 ? (int)((w >> (8 * (C.pix(edge) & 3))) & 0xffu) : 0;
    return v;
}

// Handshake over the edge (i, j) (Alg. Handshake) with the left message into i
// (Fi) and the right message into j (Bj).  Out: phi_ij (the left boundary of
// the right part) and phi_ji (the right boundary of the left part).
template <int NP, int R, bool PAD>
__device__ __forceinline__ void hs_core(const Node<NP>& ni, const Node<NP>& nj, const Taps& tp,
                                        const uint32_t (&Fi)[NP], int offF, const uint32_t (&Bj)[NP],
                                        int offB, uint32_t (&phi_ij)[NP], int& o_ij,
                                        uint32_t (&phi_ji)[NP], int& o_b, int lane, bool pad)
{
    uint32_t x[NP];
    // message j -> i
    int o_ji = offB + nj.base;
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = vadd2(nj.th[p], Bj[p]);
    msg16<NP, R, PAD>(x, phi_ji, o_ji, tp, lane, pad);
    // half of the total min-marginal at i, shared to the right: floor(m_i / 2) - phi_ji
    const int o_m = offF + ni.base + o_ji;  // even
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const uint32_t mi = vadd2(vadd2(Fi[p], ni.th[p]), phi_ji[p]);  // >= 0 in both halves
        x[p] = vsub2((mi >> 1) & 0x7fff7fffu, phi_ji[p]);
    }
    o_ij = (o_m >> 1) - o_ji;
    // keep every offset even (floor(v/2) commutes only with even shifts): an odd
    // unit moves from the offset into the vector
    const int odd = o_ij & 1;
    o_ij -= odd;
    const uint32_t oddv = splat(odd);
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = vadd2(x[p], oddv);
    msg16<NP, R, PAD>(x, phi_ij, o_ij, tp, lane, pad);
    // bounce back what cannot be shared
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = vsub2(0u, phi_ij[p]);
    o_b = -o_ij;
    msg16<NP, R, PAD>(x, phi_ji, o_b, tp, lane, pad);
}

// one Msg of a staged node into its neighbour (a sweep step in registers)
template <int NP, int R, bool PAD>
__device__ __forceinline__ void msg_from(const Node<NP>& nk, const Taps& tp, const uint32_t (&in)[NP],
                                         int in_off, uint32_t (&out)[NP], int& out_off, int lane,
                                         bool pad)
{
    uint32_t x[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = vadd2(nk.th[p], in[p]);
    out_off = in_off + nk.base;
    msg16<NP, R, PAD>(x, out, out_off, tp, lane, pad);
}

// A segment of 2-4 nodes [a, b] with boundary messages Lin, Rin: its whole
// subtree in registers (its inherited messages are recomputed from Lin/Rin,
// which gives the same values), every node finalised.  slot[0..len) hold the
// nodes a..b, staged with the edge to their right.
template <int NP, int R, bool PAD, typename DT>
__device__ __forceinline__ void leaf_block(const Dmm16Args& A, const Ctx16& C, const uint32_t* s_taps,
                                           uint8_t* const (&slot)[4], int a, int b,
                                           const uint32_t (&Lin)[NP], int oL,
                                           const uint32_t (&Rin)[NP], int oR, int lane, bool pad,
                                           long long& lb_acc)
{
    const int len = b - a + 1;
    Node<NP> n0 = read_node<NP, DT>(slot[0], C, a, lane, pad);
    Node<NP> n1 = read_node<NP, DT>(slot[1], C, len > 2 ? a + 1 : -1, lane, pad);
    uint32_t pij[NP], pji[NP];
    int oij, oji;
    if (len == 2) {
        hs_core<NP, R, PAD>(n0, n1, taps_of<R>(s_taps, n0.om), Lin, oL, Rin, oR, pij, oij, pji, oji,
                            lane, pad);
        finalise<NP, DT>(A, C, a, lane, pad, n0.th, n0.base, n0.cv, Lin, oL, pji, oji, lb_acc);
        finalise<NP, DT>(A, C, b, lane, pad, n1.th, n1.base, n1.cv, pij, oij, Rin, oR, lb_acc);
        return;
    }
    Node<NP> n2 = read_node<NP, DT>(slot[2], C, len > 3 ? a + 2 : -1, lane, pad);
    const Taps t0 = taps_of<R>(s_taps, n0.om), t1 = taps_of<R>(s_taps, n1.om);
    uint32_t F1[NP];
    int oF1;
    msg_from<NP, R, PAD>(n0, t0, Lin, oL, F1, oF1, lane, pad);  // left message into a+1
    if (len == 3) {
        // split (a+1, a+2): left part [a, a+1], right part [a+2]
        hs_core<NP, R, PAD>(n1, n2, t1, F1, oF1, Rin, oR, pij, oij, pji, oji, lane, pad);
        finalise<NP, DT>(A, C, a + 2, lane, pad, n2.th, n2.base, n2.cv, pij, oij, Rin, oR, lb_acc);
        uint32_t qij[NP], qji[NP];
        int oqij, oqji;
        hs_core<NP, R, PAD>(n0, n1, t0, Lin, oL, pji, oji, qij, oqij, qji, oqji, lane, pad);
        finalise<NP, DT>(A, C, a, lane, pad, n0.th, n0.base, n0.cv, Lin, oL, qji, oqji, lb_acc);
        finalise<NP, DT>(A, C, a + 1, lane, pad, n1.th, n1.base, n1.cv, qij, oqij, pji, oji, lb_acc);
        return;
    }
    // len == 4: split (a+1, a+2): parts [a, a+1] and [a+2, a+3]
    Node<NP> n3 = read_node<NP, DT>(slot[3], C, -1, lane, pad);
    const Taps t2 = taps_of<R>(s_taps, n2.om);
    uint32_t B2[NP];
    int oB2;
    msg_from<NP, R, PAD>(n3, t2, Rin, oR, B2, oB2, lane, pad);  // right message into a+2
    hs_core<NP, R, PAD>(n1, n2, t1, F1, oF1, B2, oB2, pij, oij, pji, oji, lane, pad);
    uint32_t qij[NP], qji[NP];
    int oqij, oqji;
    hs_core<NP, R, PAD>(n0, n1, t0, Lin, oL, pji, oji, qij, oqij, qji, oqji, lane, pad);
    finalise<NP, DT>(A, C, a, lane, pad, n0.th, n0.base, n0.cv, Lin, oL, qji, oqji, lb_acc);
    finalise<NP, DT>(A, C, a + 1, lane, pad, n1.th, n1.base, n1.cv, qij, oqij, pji, oji, lb_acc);
    hs_core<NP, R, PAD>(n2, n3, t2, pij, oij, Rin, oR, qij, oqij, qji, oqji, lane, pad);
    finalise<NP, DT>(A, C, a + 2, lane, pad, n2.th, n2.base, n2.cv, pij, oij, qji, oqji, lb_acc);
    finalise<NP, DT>(A, C, a + 3, lane, pad, n3.th, n3.base, n3.cv, qij, oqij, Rin, oR, lb_acc);
}

// One chain (row `chain` of the horizontal pass, column of the vertical pass)
// of Alg. Dual_MM's minorant computation, by the whole CTA (8 warps).  smem
// holds the taps table and the warps' staging areas.
template <int NP, int R, bool PAD, typename DT>
__device__ __forceinline__ void chain16(const Dmm16Args& A, int chain, uint8_t* smem,
                                        const uint32_t* s_taps)
{
    using G = Geo<NP, DT>;    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t* wsm = smem + 256 * kTapW * 4 + warp * G::WARP;
    uint8_t* ring = wsm;
    uint8_t* sl_i = wsm + 2 * G::BLK;
    uint8_t* sl_j = sl_i + G::NODE;
    uint8_t* sl_m0 = sl_i + 4 * G::NODE;  // boundary message of a sweep (after 4 node slots)
    uint8_t* sl_m1 = sl_m0 + G::MSG;   // inherited message of a Handshake
    Ctx16 C;
    C.which = A.which;
    C.H = A.H;
    C.W = A.W;
    C.L = A.L;
    C.n = A.which == 0 ? A.W : A.H;
    C.c = chain;
    C.KP2 = 32 * NP;
    C.c16 = A.cost16 != nullptr;
    C.err = A.err;
    const int n = C.n;
    const bool pad = PAD && (lane * 2 * NP >= A.L);
    long long lb_acc = 0;
    uint32_t zero[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) zero[p] = 0u;
    // zero boundary messages at both chain ends
    if (warp == 0) {
        store_msg<NP>(A.fmsg, A.fofs, C, 0, lane, zero, 0);
        store_msg<NP>(A.bmsg, A.bofs, C, n - 1, lane, zero, 0);
    }
    __syncthreads();

    uint8_t* const slots[4] = {sl_i, sl_j, sl_j + G::NODE, sl_j + 2 * G::NODE};
    if (n == 1) {
        if (warp == 0) {
            issue_node<NP, DT>(A, C, 0, -1, sl_i, lane);
            cp_commit();
            cp_wait<0>();
            __syncwarp();
            Node<NP> v = read_node<NP, DT>(sl_i, C, -1, lane, pad);
            finalise<NP, DT>(A, C, 0, lane, pad, v.th, v.base, v.cv, zero, 0, zero, 0, lb_acc);
        }
    } else {
        int levels = 0;
        while ((1 << levels) < n) ++levels;
        // ---- level 0: both halves swept in parallel, then the root Handshake (a
        // chain of 2-4 nodes is a single leaf block, done by the depth-first walk)
        if (n >= 5) {
            const int a = 0, b = n - 1;
            const int i = ((n + 1) >> 1) - 1, j = i + 1;
            uint32_t m[NP];
            int off = 0;
#pragma unroll
            for (int p = 0; p < NP; ++p) m[p] = 0u;
            if (warp < 2) {  // warp 0 sweeps [0, i] forward, warp 1 [j, n-1] backward
                const bool f = warp == 0;
                uint32_t* sbuf = f ? A.fmsg : A.bmsg;
                int* sofs = f ? A.fofs : A.bofs;
                sweep16<NP, R, PAD, DT>(A, C, s_taps, ring, f ? a : b, f ? 1 : -1, f ? i - a : b - j,
                                        m, off, f ? spine_fwd(a, i) : spine_bwd(j, b), sbuf, sofs,
                                        lane, pad);
                store_msg<NP>(sbuf, sofs, C, f ? i : j, lane, m, off);
            }
            __syncthreads();
            if (warp == 0) {
                issue_msg<NP>(A.fmsg, A.fofs, C, i, sl_m0, lane);
                issue_msg<NP>(A.bmsg, A.bofs, C, j, sl_m1, lane);
                issue_node<NP, DT>(A, C, i, i, sl_i, lane);
                issue_node<NP, DT>(A, C, j, -1, sl_j, lane);
                cp_commit();
                cp_wait<0>();
                __syncwarp();
                uint32_t Fi[NP], Bj[NP], pij[NP], pji[NP];
                int oF, oB, oij, oji;
                read_msg<NP>(sl_m0, lane, Fi, oF);
                read_msg<NP>(sl_m1, lane, Bj, oB);
                const Node<NP> ni = read_node<NP, DT>(sl_i, C, i, lane, pad);
                const Node<NP> nj = read_node<NP, DT>(sl_j, C, -1, lane, pad);
                hs_core<NP, R, PAD>(ni, nj, taps_of<R>(s_taps, ni.om), Fi, oF, Bj, oB, pij, oij, pji,
                                    oji, lane, pad);
                store_msg<NP>(A.bmsg, A.bofs, C, i, lane, pji, oji);  // Rin of [0, i]
                store_msg<NP>(A.fmsg, A.fofs, C, j, lane, pij, oij);  // Lin of [j, n-1]
            }
            __syncthreads();
        }
        // ---- levels 1 .. kL0-1: one warp per segment (2^level of them), a CTA
        // barrier after each level.  Then every warp walks the subtree of its
        // level-kL0 segment depth first, left child first, with no barrier: the
        // subtrees are disjoint, and a sub-chain only reads messages that its
        // ancestors left at its own positions.  Segments of 2-4 nodes are leaf
        // blocks (their whole subtree at once).
        int level = 1;
        bool dfs = n <= 4;
        uint32_t stk[32];  // a | b << 16 | right << 31 (chains of at most 8192 nodes)
        int sp = 0;
        if (dfs && warp == 0) stk[sp++] = (uint32_t)(n - 1) << 16;  // the whole chain [0, n-1]
        while (true) {
            int a = 0, b = -1;
            bool right = false;
            if (!dfs) {
                // a segment is a task only if its parent was split by a task of its own
                // (at least 5 nodes); blocks of 2-4 nodes finish their whole subtree
                int plen = 0;
                if (level >= kL0 || level >= levels) {
                    dfs = true;
                    if (levels > kL0 && segment16(n, kL0, warp, a, b, plen) && plen >= 5 && b > a)
                        stk[sp++] = (uint32_t)a | ((uint32_t)b << 16) | ((warp & 1) ? 0x80000000u : 0u);
                    continue;
                }
                if (warp < (1 << level) && segment16(n, level, warp, a, b, plen) && plen >= 5)
                    right = (warp & 1) != 0;
                else
                    b = a - 1;
            } else {
                if (sp == 0) break;
                const uint32_t e = stk[--sp];
                a = (int)(e & 0xffffu);
                b = (int)((e >> 16) & 0x7fffu);
                right = (e & 0x80000000u) != 0;
            }
            const int len = b - a + 1;
            if (len >= 2 && len <= 4) {
                __syncwarp();  // the slots of the previous task are free
                issue_msg<NP>(A.fmsg, A.fofs, C, a, sl_m0, lane);
                issue_msg<NP>(A.bmsg, A.bofs, C, b, sl_m1, lane);
                for (int k = a; k <= b; ++k) issue_node<NP, DT>(A, C, k, k < b ? k : -1, slots[k - a], lane);
                cp_commit();
                cp_wait<0>();
                __syncwarp();
                uint32_t Lin[NP], Rin[NP];
                int oL, oR;
                read_msg<NP>(sl_m0, lane, Lin, oL);
                read_msg<NP>(sl_m1, lane, Rin, oR);
                leaf_block<NP, R, PAD, DT>(A, C, s_taps, slots, a, b, Lin, oL, Rin, oR, lane, pad,
                                           lb_acc);
            } else if (len >= 5) {
                const int i = a + ((b - a + 2) >> 1) - 1, j = i + 1;
                __syncwarp();  // the slots of the previous task are free
                // boundary message of the sweep, inherited message and the two
                // Handshake nodes, staged before the sweep's own unaries
                if (right) {
                    issue_msg<NP>(A.fmsg, A.fofs, C, a, sl_m0, lane);
                    issue_msg<NP>(A.bmsg, A.bofs, C, j, sl_m1, lane);
                } else {
                    issue_msg<NP>(A.bmsg, A.bofs, C, b, sl_m0, lane);
                    issue_msg<NP>(A.fmsg, A.fofs, C, i, sl_m1, lane);
                }
                issue_node<NP, DT>(A, C, i, i, sl_i, lane);
                issue_node<NP, DT>(A, C, j, -1, sl_j, lane);
                cp_commit();
                uint32_t Fi[NP], Bj[NP], pij[NP], pji[NP];
                int oF, oB, oij, oji;
                cp_wait<0>();
                __syncwarp();
                // right child: Lin changed, the left messages are recomputed from a;
                // left child: Rin changed, the right messages are recomputed from b
                uint32_t m[NP];
                int om;
                read_msg<NP>(sl_m0, lane, m, om);
                if (right) read_msg<NP>(sl_m1, lane, Bj, oB);
                else read_msg<NP>(sl_m1, lane, Fi, oF);
                sweep16<NP, R, PAD, DT>(A, C, s_taps, ring, right ? a : b, right ? 1 : -1,
                                        right ? i - a : b - j, m, om,
                                        right ? spine_fwd(a, i) : spine_bwd(j, b),
                                        right ? A.fmsg : A.bmsg, right ? A.fofs : A.bofs, lane, pad);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    Fi[p] = right ? m[p] : Fi[p];
                    Bj[p] = right ? Bj[p] : m[p];
                }
                oF = right ? om : oF;
                oB = right ? oB : om;
                const Node<NP> ni = read_node<NP, DT>(sl_i, C, i, lane, pad);
                const Node<NP> nj = read_node<NP, DT>(sl_j, C, -1, lane, pad);
                hs_core<NP, R, PAD>(ni, nj, taps_of<R>(s_taps, ni.om), Fi, oF, Bj, oB, pij, oij,
                                    pji, oji, lane, pad);
                store_msg<NP>(A.bmsg, A.bofs, C, i, lane, pji, oji);  // Rin of [a, i]
                store_msg<NP>(A.fmsg, A.fofs, C, j, lane, pij, oij);  // Lin of [j, b]
                if (dfs) {
                    stk[sp++] = (uint32_t)j | ((uint32_t)b << 16) | 0x80000000u;
                    stk[sp++] = (uint32_t)a | ((uint32_t)i << 16);
                }
            }
            if (!dfs) {
                __syncthreads();
                ++level;
            }
        }
    }
    if (A.lb != nullptr && lane == 0 && lb_acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(A.lb), (unsigned long long)lb_acc);
}


// Launched with programmatic stream serialisation: the taps table (which no
// pass writes) is staged while the previous pass drains; everything else waits
// for that grid (griddepcontrol.wait).  Without the attribute both are no-ops.
template <int NP, int R, bool PAD, typename DT>
__global__ void __launch_bounds__(kWarps * 32, NP == 4 ? 2 : 3) dmm16_kernel(const Dmm16Args A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* s_taps = reinterpret_cast<uint32_t*>(smem);
    for (int t = threadIdx.x; t < 256 * kTapW; t += blockDim.x) s_taps[t] = A.taps16[t];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    chain16<NP, R, PAD, DT>(A, blockIdx.x, smem, s_taps);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Persistent form over the chains of many pairs of one label class: every CTA
// takes (pair, chain) tasks from a work counter, longest chains first, until
// none are left.  All pairs share the penalty (one taps table).
template <int NP, int R, bool PAD, typename DT>
__global__ void __launch_bounds__(kWarps * 32, NP == 4 ? 2 : 3)
    dmm16_batch_kernel(const __grid_constant__ Batch16Args B)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_t;
    uint32_t* s_taps = reinterpret_cast<uint32_t*>(smem);
    const uint32_t* taps = B.descs[0].taps16;
    for (int t = threadIdx.x; t < 256 * kTapW; t += blockDim.x) s_taps[t] = taps[t];
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(B.counter, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= B.n_tasks) break;
        const int2 tk = B.tasks[t];
        chain16<NP, R, PAD, DT>(B.descs[tk.x], tk.y, smem, s_taps);
        __syncthreads();
    }
}

template <int NP, typename DT>
constexpr int smem16_fixed()
{
    return 256 * kTapW * 4 + kWarps * Geo<NP, DT>::WARP;
}

// Raise a kernel's dynamic shared-memory limit to smem on the current device.
// The attribute belongs to the function on each device; `done` records, per
// device, the size already set (safe to call from several host threads).
constexpr int kMaxDevices = 64;

template <typename K>
cudaError_t ensure_smem(K kernel, int smem, std::atomic<int> (&done)[kMaxDevices])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::atomic<int>& d = done[dev < kMaxDevices ? dev : kMaxDevices - 1];
    if (d.load(std::memory_order_acquire) >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) d.store(smem, std::memory_order_release);
    return e;
}

template <int NP, int R, bool PAD, typename DT>
cudaError_t launch_one(const Dmm16Args& a, cudaStream_t s)
{
    const int smem = smem16_fixed<NP, DT>();
    static std::atomic<int> done[kMaxDevices];
    const cudaError_t e = ensure_smem(dmm16_kernel<NP, R, PAD, DT>, smem, done);
    if (e != cudaSuccess) return e;
    const int chains = a.which == 0 ? a.H : a.W;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(chains);
    cfg.blockDim = dim3(kWarps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, dmm16_kernel<NP, R, PAD, DT>, a);
}

template <int NP, int R, bool PAD, typename DT>
cudaError_t launch_batch_one(const Batch16Args& b, cudaStream_t s)
{
    const int smem = smem16_fixed<NP, DT>();
    static std::atomic<int> done[kMaxDevices];
    const cudaError_t e = ensure_smem(dmm16_batch_kernel<NP, R, PAD, DT>, smem, done);
    if (e != cudaSuccess) return e;
    dmm16_batch_kernel<NP, R, PAD, DT><<<b.grid, kWarps * 32, smem, s>>>(b);
    return cudaGetLastError();
}

template <int NP, int R, typename DT>
cudaError_t launch_r(const Dmm16Args& a, bool pad, cudaStream_t s)
{
    return pad ? launch_one<NP, R, true, DT>(a, s) : launch_one<NP, R, false, DT>(a, s);
}

template <int NP, int R, typename DT>
cudaError_t launch_batch_r(const Batch16Args& b, bool pad, cudaStream_t s)
{
    return pad ? launch_batch_one<NP, R, true, DT>(b, s) : launch_batch_one<NP, R, false, DT>(b, s);
}

}  // namespace k16

// Launchers of one (NP, DT) class; each is instantiated in its own translation unit.
template <int NP, typename DT>
cudaError_t launch16(const Dmm16Args& a, int radius, cudaStream_t s)
{
    const bool pad = a.L != 32 * 2 * NP;
    switch (radius) {
        case 1: return k16::launch_r<NP, 1, DT>(a, pad, s);
        case 2: return k16::launch_r<NP, 2, DT>(a, pad, s);
        default: return k16::launch_r<NP, 4, DT>(a, pad, s);
    }
}

template <int NP, typename DT>
cudaError_t launch16_batch(const Batch16Args& b, int radius, bool pad, cudaStream_t s)
{
    switch (radius) {
        case 1: return k16::launch_batch_r<NP, 1, DT>(b, pad, s);
        case 2: return k16::launch_batch_r<NP, 2, DT>(b, pad, s);
        default: return k16::launch_batch_r<NP, 4, DT>(b, pad, s);
    }
}

}  // namespace dm
