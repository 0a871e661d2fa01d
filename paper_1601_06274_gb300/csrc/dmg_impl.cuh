// Dual MM pass on lane groups (the default Dual MM kernel): device code,
// kernels and launchers, included by one translation unit per label class
// (dmg_g*_*.cu) so that the classes compile in parallel.
//
// Same algorithm and bit-identical results as dmm.cu and dmm16_impl.cuh --
// Alg. Dual_MM of arXiv 1601.06274 with the hierarchical minorant of App. A
// (Alg. Handshake) -- organised for the two regimes of the hierarchy:
//
// * Values.  Every message is a packed 16-bit vector plus an int32 scalar
//   offset; after each Msg the vector is shifted by an even number so that its
//   minimum is 0 or 1 (even shifts commute with the Handshake's floor(m/2)).
//   Its entries then lie in [0, P2 + 1], so messages are stored in memory as
//   one byte per label.  Duals are stored as in the one-warp kernel: an int32
//   base per pixel and uint8 or int16 deltas.
// * Two lane layouts of one message (the memory formats are the same).
//   - The top levels of the split tree are a long chain of dependent Msg
//     steps (the root sweeps half the chain) with few segments: there a whole
//     warp holds one message (LP/32 labels per lane) and the minimum over the
//     labels is one full-warp redux, for the shortest step latency.
//   - The lower levels have many segments: there a group of G = LP/16 lanes
//     holds a message (16 labels per lane, neighbours mostly in registers) and a
//     warp advances 32/G segments with one instruction stream, for the fewest
//     instructions per label.  The segments of one level have lengths q or q+1
//     (the left part of a split keeps ceil(len/2) nodes), and the split trees of
//     two segments whose lengths differ by at most one pair up node by node with
//     lengths that again differ by at most one, so the groups of a warp walk
//     their subtrees with warp-uniform control flow; a sweep that is one step
//     shorter in some group predicates that step, and the blocks of at most four
//     nodes at the bottom select their operands per group.
// * Schedule.  One CTA per chain.  The top levels run level by level (a CTA
//   barrier after each); from the level with as many segments as the CTA has
//   groups on, every group walks its segment's subtree depth first.
// * Memory.  The unaries of the next sweep steps are staged into shared memory
//   by cp.async in 16-byte chunks, two blocks of KB steps ahead.  A sweep stores
//   only the messages that a later level reads (the split points along the
//   spine it leaves behind); a Handshake stores the boundary messages of its two
//   children.

#pragma once

#include <algorithm>
#include <atomic>
#include <climits>

#include "dm_internal.cuh"

namespace dm {
namespace kg {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kInf2 = 0x3FFF3FFFu;   // 16383 in both halves: never a minimum
constexpr int KB = 4;                     // sweep steps per staged block
constexpr int RB = 3;                     // blocks in the staging ring
constexpr int kStack = 16;                // depth-first stack entries per group

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) { return __vmins2(a, b); }
__device__ __forceinline__ uint32_t vadd2(uint32_t a, uint32_t b) { return __vadd2(a, b); }
__device__ __forceinline__ uint32_t vsub2(uint32_t a, uint32_t b) { return __vsub2(a, b); }
__device__ __forceinline__ uint32_t addmin2(uint32_t a, uint32_t b, uint32_t c)
{
    return __viaddmin_s16x2(a, b, c);  // min(a + b, c) per 16-bit half
}
__device__ __forceinline__ uint32_t splat(int v) { return ((uint32_t)v & 0xffffu) * 0x10001u; }
__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xffffu); }

// One lane layout: LP labels per group (a power of two, at least 16), G lanes
// per group, DT the dual delta type, KB sweep steps per staged block.
template <int LP_, int G_, typename DT_, int KB_>
struct Lay {
    static constexpr int LP = LP_, G = G_, KB = KB_;
    using DT = DT_;
    static constexpr int LPL = LP / G;                    // labels per lane
    static constexpr int NWL = LPL / 2;                   // packed words per lane
    static_assert(NWL >= 1 && (NWL & (NWL - 1)) == 0, "1, 2, 4 or 8 packed words per lane");
};

// warps per CTA for the group layout of G lanes: 32 groups per CTA up to G = 8
// lanes, 8 warps (16 groups) for G = 16
template <int G>
constexpr int warps_of() { return G < 8 ? G : 8; }

// Shared memory of one group of the group layout: RB blocks of KB unary rows,
// KB bases and KB words holding the weights of the crossed edges, and three
// message slots.  Block 0 doubles as the four node slots of a Handshake or a
// leaf block (same layout) and blocks 1-2 as four cost rows, used only while no
// sweep is staging.  A whole-warp group uses the area of its warp's first group.
template <int LP, typename DT>
struct Area {
    static constexpr int ROW = LP * (int)sizeof(DT);
    static constexpr int BASE_AT = KB * ROW;
    static constexpr int W_AT = KB * ROW + 4 * KB;
    static constexpr int BLK = KB * ROW + 8 * KB;
    static constexpr int MSLOT = LP + 16;               // an 8-bit message and its offset
    static constexpr int GRP = RB * BLK + 3 * MSLOT;
};

// Staging geometry of a layout: a block holds KB unary rows, KB bases and KB
// words holding the weights of the crossed edges; block 0 doubles as the node
// slots of a Handshake or a leaf block.
template <class Y>
struct Geo {
    static constexpr int ROW = Y::LP * (int)sizeof(typename Y::DT);
    static constexpr int BASE_AT = Y::KB * ROW;
    static constexpr int W_AT = Y::KB * ROW + 4 * Y::KB;
    static constexpr int BLK = Y::KB * ROW + 8 * Y::KB;
};

// words per taps row in shared memory: {T1, T2, P2, valid}, then {T3, T4} for R > 2
template <int R>
constexpr int tap_words() { return R > 2 ? kTapW : 4; }

// Penalty of one edge: T_d (both halves) for d = 1..R and the cap P2.
struct Taps {
    uint32_t t[kRMax];
    int p2;
};

template <int R>
__device__ __forceinline__ Taps taps_of(const uint32_t* s_taps, int om)
{
    const uint4 v = *reinterpret_cast<const uint4*>(s_taps + om * tap_words<R>());
    Taps t;
    t.t[0] = v.x;
    t.t[1] = v.y;
    t.p2 = (int)v.z;
    if constexpr (R > 2) {
        const uint2 w = *reinterpret_cast<const uint2*>(s_taps + om * tap_words<R>() + 4);
        t.t[2] = w.x;
        t.t[3] = w.y;
    } else {
        t.t[2] = t.t[3] = 0u;
    }
    return t;
}

// A message held by a group: this lane's packed words and the offset.
template <int NWL>
struct Msg {
    uint32_t v[NWL];
    int off;
};

template <int NWL>
__device__ __forceinline__ void zero_msg(Msg<NWL>& m)
{
#pragma unroll
    for (int p = 0; p < NWL; ++p) m.v[p] = 0u;
    m.off = 0;
}

template <int NWL>
__device__ __forceinline__ void sel_msg(Msg<NWL>& d, bool take, const Msg<NWL>& s)
{
#pragma unroll
    for (int p = 0; p < NWL; ++p) d.v[p] = take ? s.v[p] : d.v[p];
    d.off = take ? s.off : d.off;
}

struct Ctx {
    int which, H, W, L, n, c;
    bool c16;        // uint16 cost volume
    int32_t* err;
    __device__ __forceinline__ int pix(int k) const { return which == 0 ? c * W + k : k * W + c; }
    // pixels between consecutive chain nodes
    __device__ __forceinline__ int pstride() const { return which == 0 ? 1 : W; }
};

// Per-lane constants of one layout.
template <class Y>
struct Lane {
    int q;            // lane within the group
    int g;            // group within the CTA (in this layout)
    bool pad;         // this lane's labels are all >= L (their unaries read as infinity)
    uint32_t s0, s1;  // byte selectors of the uint8 unpacking (pad lanes: 16383)
    uint8_t* ring;    // the group's staging ring (RB blocks of Geo<Y>::BLK bytes)
    uint8_t* ms;      // its three message slots
};

// Checked builds (-DDM_CHECKED, the library's memory-safety test) verify every
// node, edge and message position before a global access: a position outside
// the chain sets kDevErrIndex and skips the access.  Otherwise the checks
// compile away.
#ifdef DM_CHECKED
__device__ __forceinline__ bool in_chain(const Ctx& C, int k, int limit)
{
    const bool ok = k >= 0 && k < limit && C.c >= 0 && C.c < (C.which == 0 ? C.H : C.W);
    if (!ok) atomicOr(C.err, kDevErrIndex);
    return ok;
}
#else
__device__ __forceinline__ bool in_chain(const Ctx&, int, int) { return true; }
#endif

// cp.async of read-only data of the pass (unaries, bases, weights, costs): 16
// bytes bypass L1
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES)
                     : "memory");
}

// cp.async of messages this CTA wrote earlier in the pass (through L1, which
// holds the CTA's own writes)
template <int BYTES>
__device__ __forceinline__ void cp_async_ca(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// The Msg step
// ---------------------------------------------------------------------------

// minimum of v over the group's lanes: one redux for a whole warp (the
// latency-bound top levels); a butterfly of shuffles for smaller groups (the
// throughput-bound lower levels: fewer instructions than one redux per group,
// and a redux over a partial mask is slower still)
template <int G>
__device__ __forceinline__ int group_min(int v)
{
    if constexpr (G == 32) {
        return __reduce_min_sync(kFull, v);
    } else {
#pragma unroll
        for (int s = 1; s < G; s <<= 1) v = min(v, __shfl_xor_sync(kFull, v, s));
        return v;
    }
}

// packed word IDX of the group's message as seen from this lane (IDX may lie
// outside [0, NWL): the words of the lanes to the left or right; 16383 past the
// group's ends)
template <int G, int NWL, int IDX>
__device__ __forceinline__ uint32_t ext_word(const uint32_t (&x)[NWL], int q)
{
    constexpr int off = IDX >= 0 ? IDX / NWL : -((-IDX + NWL - 1) / NWL);
    constexpr int loc = IDX - off * NWL;
    if constexpr (off == 0) {
        return x[loc];
    } else if constexpr (G == 1 || off >= G || -off >= G) {
        return kInf2;
    } else if constexpr (off < 0) {
        const uint32_t v = __shfl_up_sync(kFull, x[loc], -off, G);
        return q + off >= 0 ? v : kInf2;
    } else {
        const uint32_t v = __shfl_down_sync(kFull, x[loc], off, G);
        return q + off <= G - 1 ? v : kInf2;
    }
}

template <int G, int NWL, int HH, int IDX>
__device__ __forceinline__ void fill_ext(const uint32_t (&x)[NWL], uint32_t (&E)[NWL + 2 * HH], int q)
{
    if constexpr (IDX < NWL + HH) {
        E[IDX + HH] = ext_word<G, NWL, IDX>(x, q);
        fill_ext<G, NWL, HH, IDX + 1>(x, E, q);
    }
}

// out = Msg(x) normalised; the shift goes into off.
//   Msg(a)(x') = min(a(x'), min_{d <= R} min(a(x'-d), a(x'+d)) + T_d, min a + P2)
template <int G, int NWL, int R>
__device__ __forceinline__ void msg_core(const uint32_t (&x)[NWL], uint32_t (&out)[NWL], int& off,
                                         const Taps& tp, int q)
{
    constexpr int HH = (R + 1) / 2;
    uint32_t t[NWL];
#pragma unroll
    for (int p = 0; p < NWL; ++p) t[p] = x[p];
#pragma unroll
    for (int s = 1; s < NWL; s <<= 1)
#pragma unroll
        for (int p = 0; p + s < NWL; p += 2 * s) t[p] = vmin2(t[p], t[p + s]);
    const int m = group_min<G>(min(lo16(t[0]), (int)t[0] >> 16));
    uint32_t E[NWL + 2 * HH];
    fill_ext<G, NWL, HH, -HH>(x, E, q);
    const int shift = m & ~1;                        // even floor of the minimum
    const uint32_t negs = splat(-shift);
    const uint32_t caps = splat(m - shift + tp.p2);  // (min x + P2) - shift
#pragma unroll
    for (int p = 0; p < NWL; ++p) {
        uint32_t res = x[p];
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            uint32_t l, r;
            if (d & 1) {  // labels (2p-d, 2p+1-d) and (2p+d, 2p+1+d) straddle two words
                l = __byte_perm(E[p - (d + 1) / 2 + HH], E[p - (d - 1) / 2 + HH], 0x5432);
                r = __byte_perm(E[p + (d - 1) / 2 + HH], E[p + (d + 1) / 2 + HH], 0x5432);
            } else {
                l = E[p - d / 2 + HH];
                r = E[p + d / 2 + HH];
            }
            res = addmin2(vmin2(l, r), tp.t[d - 1], res);
        }
        out[p] = addmin2(res, negs, caps);  // min(res, min x + P2) - shift
    }
    off += shift;
}

// ---------------------------------------------------------------------------
// Rows and messages between memory and registers
// ---------------------------------------------------------------------------

// N bytes at p (N in {2, 4, 8, 16, 32}, aligned to min(N, 16)) as little-endian words
template <int N>
__device__ __forceinline__ void load_bytes(const uint8_t* p, uint32_t (&w)[(N + 3) / 4])
{
    if constexpr (N == 32) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint4 u = *reinterpret_cast<const uint4*>(p + 16);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        w[4] = u.x; w[5] = u.y; w[6] = u.z; w[7] = u.w;
    } else if constexpr (N == 16) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (N == 8) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (N == 4) {
        w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else {
        w[0] = *reinterpret_cast<const uint16_t*>(p);
    }
}

template <int N>
__device__ __forceinline__ void store_bytes(uint8_t* p, const uint32_t (&w)[(N + 3) / 4])
{
    if constexpr (N == 32) {
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(p + 16) = make_uint4(w[4], w[5], w[6], w[7]);
    } else if constexpr (N == 16) {
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (N == 8) {
        *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    } else if constexpr (N == 4) {
        *reinterpret_cast<uint32_t*>(p) = w[0];
    } else {
        *reinterpret_cast<uint16_t*>(p) = (uint16_t)w[0];
    }
}

// this lane's labels of a staged unary row as packed pairs; pad lanes read
// 16383 (uint8 rows: the byte selectors pick it from the constant operand)
template <class Y>
__device__ __forceinline__ void read_row(const uint8_t* row, const Lane<Y>& ln, uint32_t (&th)[Y::NWL])
{
    if constexpr (sizeof(typename Y::DT) == 1) {
        uint32_t w[(Y::LPL + 3) / 4];
        load_bytes<Y::LPL>(row + ln.q * Y::LPL, w);
#pragma unroll
        for (int p = 0; p < Y::NWL; ++p) th[p] = __byte_perm(w[p >> 1], 0x00003FFFu, (p & 1) ? ln.s1 : ln.s0);
    } else {
        uint32_t w[(2 * Y::LPL + 3) / 4];
        load_bytes<2 * Y::LPL>(row + ln.q * 2 * Y::LPL, w);
#pragma unroll
        for (int p = 0; p < Y::NWL; ++p) th[p] = ln.pad ? kInf2 : w[p];
    }
}

// 8-bit stored labels (entries in [0, 255]) <-> packed pairs
template <int NWL>
__device__ __forceinline__ void unpack_u8(const uint32_t (&w)[(2 * NWL + 3) / 4], uint32_t (&m)[NWL])
{
#pragma unroll
    for (int p = 0; p < NWL; ++p) m[p] = __byte_perm(w[p >> 1], 0, (p & 1) ? 0x4342 : 0x4140);
}

template <int NWL>
__device__ __forceinline__ void pack_u8(const uint32_t (&m)[NWL], uint32_t (&w)[(2 * NWL + 3) / 4])
{
    if constexpr (NWL == 1) {
        w[0] = __byte_perm(m[0], 0, 0x4420);
    } else {
#pragma unroll
        for (int k = 0; k < NWL / 2; ++k) w[k] = __byte_perm(m[2 * k], m[2 * k + 1], 0x6420);
    }
}

template <class Y>
__device__ __forceinline__ void store_msg(uint8_t* buf, int32_t* ofs, const Ctx& C, int pos,
                                          const Lane<Y>& ln, const Msg<Y::NWL>& m, bool active)
{
    if (!active || !in_chain(C, pos, C.n)) return;
    const size_t node = (size_t)C.c * C.n + pos;
    uint32_t w[(2 * Y::NWL + 3) / 4];
    pack_u8<Y::NWL>(m.v, w);
    store_bytes<Y::LPL>(buf + node * Y::LP + ln.q * Y::LPL, w);
    if (ln.q == 0) ofs[node] = m.off;
}

template <class Y>
__device__ __forceinline__ void load_msg(const uint8_t* buf, const int32_t* ofs, const Ctx& C, int pos,
                                         const Lane<Y>& ln, Msg<Y::NWL>& m, bool active)
{
    if (!active || !in_chain(C, pos, C.n)) {
        zero_msg(m);
        return;
    }
    const size_t node = (size_t)C.c * C.n + pos;
    uint32_t w[(2 * Y::NWL + 3) / 4];
    load_bytes<Y::LPL>(buf + node * Y::LP + ln.q * Y::LPL, w);
    unpack_u8<Y::NWL>(w, m.v);
    m.off = ofs[node];
}

// message slots of the group
template <class Y>
__device__ __forceinline__ uint8_t* mslot(const Lane<Y>& ln, int i)
{
    return ln.ms + i * Area<Y::LP, typename Y::DT>::MSLOT;
}

// stage message `pos` of (buf, ofs) into message slot `slot` (cp.async, the
// group's lanes over its 16-byte chunks)
template <class Y>
__device__ __forceinline__ void issue_msg(const uint8_t* buf, const int32_t* ofs, const Ctx& C, int pos,
                                          const Lane<Y>& ln, int slot, bool active)
{
    if (!active || !in_chain(C, pos, C.n)) return;
    const size_t node = (size_t)C.c * C.n + pos;
    uint8_t* d = mslot(ln, slot);
    for (int t = ln.q; t < Y::LP / 16; t += Y::G) cp_async_ca<16>(d + 16 * t, buf + node * Y::LP + 16 * t);
    if (ln.q == 0) cp_async_ca<4>(d + Y::LP, ofs + node);
}

template <class Y>
__device__ __forceinline__ void read_msg_slot(const Lane<Y>& ln, int slot, Msg<Y::NWL>& m, bool active)
{
    const uint8_t* d = mslot(ln, slot);
    uint32_t w[(2 * Y::NWL + 3) / 4];
    load_bytes<Y::LPL>(d + ln.q * Y::LPL, w);
    unpack_u8<Y::NWL>(w, m.v);
    m.off = *reinterpret_cast<const int*>(d + Y::LP);
    if (!active) zero_msg(m);
}

// write a message into message slot `slot`
template <class Y>
__device__ __forceinline__ void put_msg_slot(const Lane<Y>& ln, int slot, const Msg<Y::NWL>& m)
{
    uint8_t* d = mslot(ln, slot);
    uint32_t w[(2 * Y::NWL + 3) / 4];
    pack_u8<Y::NWL>(m.v, w);
    store_bytes<Y::LPL>(d + ln.q * Y::LPL, w);
    if (ln.q == 0) *reinterpret_cast<int*>(d + Y::LP) = m.off;
    __syncwarp();
}

// Stage cnt nodes k0, k0 + dir, ... into a block laid out like Area::BLK:
// unary rows in 16-byte chunks over the group's lanes (chunks past the L labels
// of the row skipped), then the bases and the words holding the weights of the
// edges the steps cross (`wdir`: (k, k+1) for +1, (k-1, k) for -1).
template <class Y>
__device__ __forceinline__ void issue_nodes(const Dmm16Args& A, const Ctx& C, int k0, int dir, int cnt,
                                            int wdir, uint8_t* blk, const Lane<Y>& ln)
{
    using DT = typename Y::DT;
    using Gm = Geo<Y>;
    constexpr int CH = Gm::ROW / 16;  // chunks per staged row (a power of two)
    const int rowd = C.L * (int)sizeof(DT);
    const long long step = (long long)dir * C.pstride() * rowd;
    const uint8_t* src = reinterpret_cast<const uint8_t*>(A.delta_in) + (long long)C.pix(k0) * rowd;
    for (int t = ln.q; t < cnt * CH; t += Y::G) {
        const int u = t / CH, c = t & (CH - 1);
        if (c * 16 < rowd && in_chain(C, k0 + dir * u, C.n))
            cp_async<16>(blk + u * Gm::ROW + c * 16, src + u * step + c * 16);
    }
    for (int t = ln.q; t < 2 * cnt; t += Y::G) {
        const int u = t >> 1;
        const int k = k0 + dir * u;
        if ((t & 1) == 0) {
            if (in_chain(C, k, C.n)) cp_async<4>(blk + Gm::BASE_AT + 4 * u, A.base_in + C.pix(k));
        } else {
            const int e = wdir > 0 ? k : k - 1;
            if (e >= 0 && e < C.n - 1 && in_chain(C, e, C.n - 1))
                cp_async<4>(blk + Gm::W_AT + 4 * u, A.wedge + (C.pix(e) & ~3));
        }
    }
}

__device__ __forceinline__ int omega_of(uint32_t word, const Ctx& C, int e)
{
    return e >= 0 ? (int)((word >> (8 * (C.pix(e) & 3))) & 0xffu) : 0;
}

// The messages a sweep must leave behind: forward over [a, i] (D = i - a
// steps) the split points a + (D >> t), t >= 1, while D >> t >= 1; backward
// over [j, b] (E = b - j + 1 nodes) the nodes b + 1 - (E >> t) while
// E >> t >= 2.  Both are reached with t decreasing.
struct Spine {
    int t, base, span, dir;
    __device__ __forceinline__ int pos() const
    {
        if (t <= 0) return -0x40000000;
        return dir > 0 ? base + (span >> t) : base + 1 - (span >> t);
    }
};

__device__ __forceinline__ Spine spine_fwd(int a, int i)
{
    Spine sp{0, a, i - a, +1};
    while ((sp.span >> (sp.t + 1)) >= 1) ++sp.t;
    return sp;
}

__device__ __forceinline__ Spine spine_bwd(int j, int b)
{
    Spine sp{0, b, b - j + 1, -1};
    while ((sp.span >> (sp.t + 1)) >= 2) ++sp.t;
    return sp;
}

// ---------------------------------------------------------------------------
// Sweeps, Handshakes, leaf blocks
// ---------------------------------------------------------------------------

// One sweep per group: cnt_g Msg steps from node k0 in direction dir (+1:
// forward, messages enter k0+1, k0+2, ...; -1: backward).  m holds the boundary
// message on entry and the last message on exit; the messages that enter the
// spine positions are stored.  Counts differ by at most one over the warp
// (minc, maxc their extremes); only the one step from minc on is predicated.
// Every lane's share of a block's copies is fixed for the sweep: the same
// chunks of the same rows, one block further on each time.
//
// `extra` more nodes past the last step are staged as well (the Handshake's two
// nodes; they stay in the ring at sweep positions cnt_g and cnt_g + 1), and the
// boundary message is read from message slot `mslot_in` after the first block
// arrives (its copy must be committed before the call).
template <class Y, int R>
__device__ __forceinline__ void sweep(const Dmm16Args& A, const Ctx& C, const uint32_t* s_taps,
                                      const Lane<Y>& ln, int k0, int dir, int cnt_g, int minc, int maxc,
                                      int extra, int mslot_in, bool active, Msg<Y::NWL>& m, Spine sp)
{
    using DT = typename Y::DT;
    using Gm = Geo<Y>;
    constexpr int NWL = Y::NWL, KBY = Y::KB, CH = Gm::ROW / 16;
    uint8_t* sbuf = dir > 0 ? reinterpret_cast<uint8_t*>(A.fmsg) : reinterpret_cast<uint8_t*>(A.bmsg);
    int32_t* sofs = dir > 0 ? A.fofs : A.bofs;
    const int nblk = (maxc + KBY - 1) / KBY;              // blocks with steps
    const int nstg = (maxc + extra + KBY - 1) / KBY;      // blocks to stage
    const int stg_g = active ? cnt_g + extra : 0;         // this group's staged nodes
    // copy plan: node u of block bi is node k0 + dir (KBY bi + u), pixel pix0 + pst (KBY bi + u)
    const int rowd = C.L * (int)sizeof(DT);
    const int pix0 = C.pix(k0);
    const int pst = dir * C.pstride();
    const long long rstep = (long long)pst * rowd;
    const uint8_t* rsrc = reinterpret_cast<const uint8_t*>(A.delta_in) + (long long)pix0 * rowd;
    const int wsh = dir > 0 ? 0 : C.pstride();  // the crossed edge (k, k+1) or (k-1, k) by its left pixel
    auto issue = [&](int bi) {
        const int cb = min(KBY, stg_g - bi * KBY);
        if (bi >= nstg || cb <= 0) return;
        uint8_t* blk = ln.ring + (bi % RB) * Gm::BLK;
        const uint8_t* src = rsrc + (long long)bi * KBY * rstep;
#pragma unroll
        for (int t = ln.q; t < KBY * CH; t += Y::G) {
            const int u = t / CH, c = t & (CH - 1);
            if (u < cb && c * 16 < rowd && in_chain(C, k0 + dir * (bi * KBY + u), C.n))
                cp_async<16>(blk + u * Gm::ROW + c * 16, src + u * rstep + c * 16);
        }
        for (int t = ln.q; t < 2 * cb; t += Y::G) {
            const int u = t >> 1;
            const int px = pix0 + pst * (bi * KBY + u);
            const int k = k0 + dir * (bi * KBY + u);
            if ((t & 1) == 0) {
                if (in_chain(C, k, C.n)) cp_async<4>(blk + Gm::BASE_AT + 4 * u, A.base_in + px);
            } else {
                const int e = dir > 0 ? k : k - 1;  // the crossed edge (a staged extra node may have none)
                if (e >= 0 && e < C.n - 1 && in_chain(C, e, C.n - 1))
                    cp_async<4>(blk + Gm::W_AT + 4 * u, A.wedge + ((px - wsh) & ~3));
            }
        }
    };
    __syncwarp();  // the ring's previous contents are consumed
#pragma unroll 1
    for (int bi = 0; bi < RB - 1; ++bi) {  // RB - 1 commit groups, some possibly empty
        issue(bi);
        cp_commit();
    }
    if (nblk == 0) {  // no step: the staged nodes and the boundary message only
        cp_wait<0>();
        __syncwarp();
        if (mslot_in >= 0) read_msg_slot(ln, mslot_in, m, active);
        return;
    }
    // the step after which the next spine message is stored (its message enters
    // node k0 + dir (step + 1)); steps run in stretches that end at a spine
    // store or a block's end, with no other test inside a stretch
    auto store_step = [&]() {
        const int pos = sp.pos();
        return pos < -0x10000000 ? 0x3fffffff : (dir > 0 ? pos - k0 - 1 : k0 - 1 - pos);
    };
    int sstep = store_step();
    const int wshift = dir > 0 ? 0 : C.pstride();
    Taps tp;
#pragma unroll 1
    for (int bi = 0; bi < nblk; ++bi) {
        cp_wait<RB - 2>();
        __syncwarp();
        if (bi == 0 && mslot_in >= 0) read_msg_slot(ln, mslot_in, m, active);
        const uint8_t* blk = ln.ring + (bi % RB) * Gm::BLK;
        const int s0 = bi * KBY;
        const int steps = min(KBY, maxc - s0);
        const int plain = min(steps, max(0, minc - s0));  // steps every group takes
        // a step's row and base, and its penalty taps, loaded one step ahead; the
        // word holding the edge weight two steps ahead, so that the taps lookup
        // (which indexes by the weight) does not wait on a fresh load
        uint32_t th[NWL];
        read_row<Y>(blk, ln, th);
        int base = *reinterpret_cast<const int*>(blk + Gm::BASE_AT);
        int px = pix0 + pst * s0 - wshift;  // left pixel of the step's edge
        tp = taps_of<R>(s_taps, (int)((*reinterpret_cast<const uint32_t*>(blk + Gm::W_AT) >> (8 * (px & 3))) & 0xffu));
        uint32_t ww_n = *reinterpret_cast<const uint32_t*>(blk + Gm::W_AT + 4 * min(1, KBY - 1));
        int u = 0;
        int stretches = 0;
#pragma unroll 1
        while (u < plain) {
            // warp-uniform: the groups of a warp store their spine messages at
            // different steps; each stretch ends at the earliest of them
            const int stop = __reduce_min_sync(kFull, min(plain, sstep - s0 + 1));
            if (stop <= u || ++stretches > KBY + 1) {  // cannot happen: report it rather than spin
                if (ln.q == 0) atomicOr(C.err, kDevErrIndex);
                break;
            }
#pragma unroll 1
            for (; u < stop; ++u) {
                uint32_t x[NWL];
#pragma unroll
                for (int p = 0; p < NWL; ++p) x[p] = th[p] + m.v[p];  // < 2^15 per half: no carry
                m.off += base;
                const Taps tc = tp;
                {  // the next step's inputs (the last row again at the block's end)
                    const int un = min(u + 1, KBY - 1);
                    read_row<Y>(blk + un * Gm::ROW, ln, th);
                    base = *reinterpret_cast<const int*>(blk + Gm::BASE_AT + 4 * un);
                    px += pst;
                    tp = taps_of<R>(s_taps, (int)((ww_n >> (8 * (px & 3))) & 0xffu));
                    ww_n = *reinterpret_cast<const uint32_t*>(blk + Gm::W_AT + 4 * min(u + 2, KBY - 1));
                }
                msg_core<Y::G, NWL, R>(x, m.v, m.off, tc, ln.q);
            }
            if (s0 + u - 1 == sstep) {  // the message entering the spine position
                store_msg<Y>(sbuf, sofs, C, k0 + dir * (sstep + 1), ln, m, sstep < cnt_g);
                --sp.t;
                sstep = store_step();
            }
        }
        if (u < steps) {
            // the one step that some groups do not take (the last of the sweep)
            const int s = s0 + u;
            uint32_t x[NWL];
#pragma unroll
            for (int p = 0; p < NWL; ++p) x[p] = th[p] + m.v[p];
            Msg<NWL> o;
            o.off = m.off + base;
            msg_core<Y::G, NWL, R>(x, o.v, o.off, tp, ln.q);
            sel_msg(m, s < cnt_g, o);
            if (s == sstep) {
                store_msg<Y>(sbuf, sofs, C, k0 + dir * (s + 1), ln, m, s < cnt_g);
                --sp.t;
                sstep = store_step();
            }
        }
        __syncwarp();
        issue(bi + RB - 1);
        cp_commit();
    }
    cp_wait<0>();
}

// Stage nodes a .. a+cnt-1 into the node slots (block 0 of the area: unary
// rows, bases, the weights of the edges to their right) and, with `cost`, their
// cost rows after block 0 (cnt <= 4; blocks 1-2 hold four uint16 rows).
template <class Y>
__device__ __forceinline__ void stage_slots(const Dmm16Args& A, const Ctx& C, const Lane<Y>& ln, int a,
                                            int cnt, bool cost)
{
    using Gm = Geo<Y>;
    __syncwarp();
    issue_nodes<Y>(A, C, a, 1, cnt, 1, ln.ring, ln);
    if (cost) {
        const int cb = C.c16 ? 2 : 1;
        const int crow = Y::LP * cb;     // staged cost row
        const int chunks = crow / 16;    // a power of two
        const int rowc = C.L * cb;
        const uint8_t* src = C.c16 ? reinterpret_cast<const uint8_t*>(A.cost16) : A.cost;
        for (int t = ln.q; t < cnt * chunks; t += Y::G) {
            const int u = t / chunks, c = t & (chunks - 1);
            if (c * 16 < rowc && in_chain(C, a + u, C.n))
                cp_async<16>(ln.ring + Gm::BLK + u * crow + c * 16,
                             src + (size_t)C.pix(a + u) * rowc + c * 16);
        }
    }
    cp_commit();
}

template <class Y>
__device__ __forceinline__ int slot_omega(const Lane<Y>& ln, int i, const Ctx& C, int e)
{
    return omega_of(*reinterpret_cast<const uint32_t*>(ln.ring + Geo<Y>::W_AT + 4 * i), C, e);
}

template <class Y>
__device__ __forceinline__ int slot_base(const Lane<Y>& ln, int i)
{
    return *reinterpret_cast<const int*>(ln.ring + Geo<Y>::BASE_AT + 4 * i);
}

// Handshake over the edge (i, j) (Alg. Handshake) with the left message into i
// (F) and the right message into j (B); the staged unary rows and bases of i
// and j are given.  Out: phi_ij (the left boundary message of the right part)
// and phi_ji (the right boundary message of the left part).
template <class Y, int R>
__device__ __forceinline__ void handshake_at(const Lane<Y>& ln, const uint8_t* row_i, int base_i,
                                             const uint8_t* row_j, int base_j, const Taps& tp,
                                             const Msg<Y::NWL>& F, const Msg<Y::NWL>& B, Msg<Y::NWL>& pij,
                                             Msg<Y::NWL>& pji)
{
    constexpr int NWL = Y::NWL;
    uint32_t x[NWL];
    // message j -> i
    Msg<NWL> p1;
    read_row<Y>(row_j, ln, x);
    p1.off = B.off + base_j;
#pragma unroll
    for (int p = 0; p < NWL; ++p) x[p] += B.v[p];
    msg_core<Y::G, NWL, R>(x, p1.v, p1.off, tp, ln.q);
    // half of the total min-marginal at i, shared to the right: floor(m_i / 2) - phi_ji
    read_row<Y>(row_i, ln, x);
    const int o_m = F.off + base_i + p1.off;  // even
#pragma unroll
    for (int p = 0; p < NWL; ++p) {
        const uint32_t mi = F.v[p] + x[p] + p1.v[p];  // >= 0 and < 2^15 in both halves
        x[p] = vsub2((mi >> 1) & 0x7fff7fffu, p1.v[p]);
    }
    pij.off = (o_m >> 1) - p1.off;
    // keep every offset even (floor(v/2) commutes only with even shifts): an odd
    // unit moves from the offset into the vector
    const int odd = pij.off & 1;
    pij.off -= odd;
    const uint32_t oddv = splat(odd);
#pragma unroll
    for (int p = 0; p < NWL; ++p) x[p] = vadd2(x[p], oddv);
    msg_core<Y::G, NWL, R>(x, pij.v, pij.off, tp, ln.q);
    // bounce back what cannot be shared (labels of pad lanes stay out of the minimum)
#pragma unroll
    for (int p = 0; p < NWL; ++p) x[p] = ln.pad ? kInf2 : vsub2(0u, pij.v[p]);
    pji.off = -pij.off;
    msg_core<Y::G, NWL, R>(x, pji.v, pji.off, tp, ln.q);
}

// the same with the nodes staged in the node slots si, sj
template <class Y, int R>
__device__ __forceinline__ void handshake(const Lane<Y>& ln, int si, int sj, const Taps& tp,
                                          const Msg<Y::NWL>& F, const Msg<Y::NWL>& B, Msg<Y::NWL>& pij,
                                          Msg<Y::NWL>& pji)
{
    using Gm = Geo<Y>;
    handshake_at<Y, R>(ln, ln.ring + si * Gm::ROW, slot_base(ln, si), ln.ring + sj * Gm::ROW, slot_base(ln, sj),
                       tp, F, B, pij, pji);
}

// one Msg of a staged node's unary plus an incoming message (a sweep step in registers)
template <class Y, int R>
__device__ __forceinline__ void msg_from(const Lane<Y>& ln, int si, const Taps& tp, const Msg<Y::NWL>& in,
                                         Msg<Y::NWL>& out)
{
    uint32_t x[Y::NWL];
    read_row<Y>(ln.ring + si * Geo<Y>::ROW, ln, x);
#pragma unroll
    for (int p = 0; p < Y::NWL; ++p) x[p] += in.v[p];
    out.off = in.off + slot_base(ln, si);
    msg_core<Y::G, Y::NWL, R>(x, out.v, out.off, tp, ln.q);
}

// Output of a node that is a single node of the hierarchy: it keeps
// theta + Lin + Rin.  Both passes store c + Lin + Rin (the horizontal pass's
// lambda_h = c + lambda_v + Lin + Rin - lambda_v; the vertical pass's
// c + lambda_v, the next horizontal unary), base = Lin.off + Rin.off; with
// labels or lb set (the last vertical pass) the label is argmin_l of
// theta + Lin + Rin (ties to the smallest label) and the node adds its minimum
// to the group's lower-bound sum.  Node k is staged in slot i (unary, base,
// cost row).  All lanes compute; `active` gates the stores.
template <class Y>
__device__ __forceinline__ void finalise(const Dmm16Args& A, const Ctx& C, const Lane<Y>& ln, int i,
                                         int k, const Msg<Y::NWL>& lin, const Msg<Y::NWL>& rin,
                                         long long* s_lb, bool active)
{
    using DT = typename Y::DT;
    using Gm = Geo<Y>;
    constexpr int NWL = Y::NWL;
    active = active && in_chain(C, k, C.n);
    const int pix = C.pix(k < 0 ? 0 : (k >= C.n ? C.n - 1 : k));
    uint32_t v[NWL];
    {
        uint32_t cv[NWL];
        const uint8_t* crow = ln.ring + Gm::BLK;
        if (C.c16) {
            uint32_t w[(2 * Y::LPL + 3) / 4];
            load_bytes<2 * Y::LPL>(crow + i * 2 * Y::LP + ln.q * 2 * Y::LPL, w);
#pragma unroll
            for (int p = 0; p < NWL; ++p) cv[p] = w[p];
        } else {
            uint32_t w[(Y::LPL + 3) / 4];
            load_bytes<Y::LPL>(crow + i * Y::LP + ln.q * Y::LPL, w);
            unpack_u8<NWL>(w, cv);
        }
#pragma unroll
        for (int p = 0; p < NWL; ++p) v[p] = vadd2(vadd2(lin.v[p], rin.v[p]), cv[p]);
    }
    if (active && ln.q == 0) A.base_out[pix] = lin.off + rin.off;
    if (active && !ln.pad) {
        if constexpr (sizeof(DT) == 1) {
            // every delta is in [0, 255]: the host only picks 8-bit storage when it must be
            uint32_t bad = 0;
#pragma unroll
            for (int p = 0; p < NWL; ++p) bad |= v[p];
            if (bad & 0xff00ff00u) atomicOr(A.err, kDevErrRange);
            uint32_t w[(2 * NWL + 3) / 4];
            pack_u8<NWL>(v, w);
            store_bytes<Y::LPL>(reinterpret_cast<uint8_t*>(A.delta_out) + (size_t)pix * C.L + ln.q * Y::LPL, w);
        } else {
            uint8_t* dp = reinterpret_cast<uint8_t*>(reinterpret_cast<int16_t*>(A.delta_out) + (size_t)pix * C.L +
                                                     ln.q * Y::LPL);
            store_bytes<2 * Y::LPL>(dp, v);
        }
    }
    if (A.labels != nullptr || A.lb != nullptr) {
        uint32_t th[NWL];
        read_row<Y>(ln.ring + i * Gm::ROW, ln, th);
        const int th_base = slot_base(ln, i);
        // key = value * 512 + label: the minimum is the smallest value, ties to the smallest label
        int key = INT_MAX;
        if (!ln.pad) {
#pragma unroll
            for (int p = 0; p < NWL; ++p) {
                const uint32_t nu = vadd2(vadd2(lin.v[p], rin.v[p]), th[p]);
                const int l0 = ln.q * Y::LPL + 2 * p;
                key = min(key, min(lo16(nu) * 512 + l0, ((int)nu >> 16) * 512 + l0 + 1));
            }
        }
        key = group_min<Y::G>(key);
        if (active && ln.q == 0) {
            if (A.labels != nullptr) A.labels[pix] = (uint16_t)(key & 511);
            *s_lb += (long long)(key >> 9) + th_base + lin.off + rin.off;
        }
    }
}

// A block of at most four nodes [a, b] (len = b - a + 1 in 0..4 per group,
// lengths differing by at most one over the warp, maxlen their maximum) whose
// boundary messages Lin and Rin are stored at fmsg[a] and bmsg[b] (or are zero
// at the chain ends): its whole subtree at once, every node finalised.  Lin,
// Rin and phi_ji wait in the group's message slots 0-2 between their uses.
template <class Y, int R>
__device__ __forceinline__ void leaf_block(const Dmm16Args& A, const Ctx& C, const uint32_t* s_taps,
                                           const Lane<Y>& ln, int a, int len, int maxlen, long long* s_lb)
{
    using M = Msg<Y::NWL>;
    const uint8_t* fm = reinterpret_cast<const uint8_t*>(A.fmsg);
    const uint8_t* bm = reinterpret_cast<const uint8_t*>(A.bmsg);
    stage_slots<Y>(A, C, ln, a, len, true);
    issue_msg<Y>(fm, A.fofs, C, a, ln, 0, len >= 1);
    issue_msg<Y>(bm, A.bofs, C, a + len - 1, ln, 1, len >= 1);
    cp_commit();
    cp_wait<0>();
    __syncwarp();
    const bool any = len >= 1;
    M lin, rin;
    if (maxlen == 1) {
        read_msg_slot(ln, 0, lin, any);
        read_msg_slot(ln, 1, rin, any);
        finalise(A, C, ln, 0, a, lin, rin, s_lb, len == 1);
        return;
    }
    const Taps tp0 = taps_of<R>(s_taps, slot_omega(ln, 0, C, a));
    M pij, pji;
    if (maxlen == 2) {
        // len 2: Handshake (a, a+1); len 1: node a alone
        const bool two = len == 2;
        read_msg_slot(ln, 0, lin, any);
        read_msg_slot(ln, 1, rin, any);
        handshake<Y, R>(ln, 0, 1, tp0, lin, rin, pij, pji);
        finalise(A, C, ln, 1, a + 1, pij, rin, s_lb, two);
        sel_msg(pji, !two, rin);
        finalise(A, C, ln, 0, a, lin, pji, s_lb, any);
        return;
    }
    const Taps tp1 = taps_of<R>(s_taps, slot_omega(ln, 1, C, a + 1));
    if (maxlen == 3) {
        // len 3: F1 = Msg(node a + Lin); Handshake (a+1, a+2) with (F1, Rin); node
        //        a+2 keeps (phi_ij, Rin); Handshake (a, a+1) with (Lin, phi_ji).
        // len 2: Handshake (a, a+1) with (Lin, Rin).
        const bool three = len == 3;
        {
            M F1;
            read_msg_slot(ln, 0, lin, any);
            msg_from<Y, R>(ln, 0, tp0, lin, F1);
            sel_msg(F1, !three, lin);
            read_msg_slot(ln, 1, rin, any);
            handshake<Y, R>(ln, three ? 1 : 0, three ? 2 : 1, three ? tp1 : tp0, F1, rin, pij, pji);
        }
        // the right part's single node: a+2 (len 3) or a+1 (len 2)
        finalise(A, C, ln, three ? 2 : 1, a + (three ? 2 : 1), pij, rin, s_lb, len >= 2);
        put_msg_slot(ln, 2, pji);
        M qij, qji;
        read_msg_slot(ln, 0, lin, any);
        handshake<Y, R>(ln, 0, 1, tp0, lin, pji, qij, qji);
        read_msg_slot(ln, 2, pji, any);
        finalise(A, C, ln, 1, a + 1, qij, pji, s_lb, three);
        sel_msg(qji, !three, pji);
        read_msg_slot(ln, 0, lin, any);
        finalise(A, C, ln, 0, a, lin, qji, s_lb, len >= 2);
        return;
    }
    // maxlen == 4: lengths 3 or 4
    // len 4: F1 = Msg(a + Lin), B2 = Msg(a+3 + Rin); Handshake (a+1, a+2) with (F1, B2);
    //        then [a+2, a+3] with (phi_ij, Rin) and [a, a+1] with (Lin, phi_ji).
    // len 3: F1; Handshake (a+1, a+2) with (F1, Rin); node a+2 = (phi_ij, Rin);
    //        then [a, a+1] with (Lin, phi_ji).
    const bool four = len == 4;
    const Taps tp2 = taps_of<R>(s_taps, slot_omega(ln, 2, C, four ? a + 2 : -1));
    {
        M F1, B2;
        read_msg_slot(ln, 0, lin, any);
        msg_from<Y, R>(ln, 0, tp0, lin, F1);
        read_msg_slot(ln, 1, rin, any);
        msg_from<Y, R>(ln, 3, tp2, rin, B2);
        sel_msg(B2, !four, rin);
        handshake<Y, R>(ln, 1, 2, tp1, F1, B2, pij, pji);
    }
    put_msg_slot(ln, 2, pji);
    {
        M rij, rji;
        read_msg_slot(ln, 1, rin, any);
        handshake<Y, R>(ln, 2, 3, tp2, pij, rin, rij, rji);
        finalise(A, C, ln, 3, a + 3, rij, rin, s_lb, four);
        sel_msg(rji, !four, rin);
        finalise(A, C, ln, 2, a + 2, pij, rji, s_lb, len >= 3);
    }
    M qij, qji;
    read_msg_slot(ln, 0, lin, any);
    read_msg_slot(ln, 2, pji, any);
    handshake<Y, R>(ln, 0, 1, tp0, lin, pji, qij, qji);
    read_msg_slot(ln, 2, pji, any);
    finalise(A, C, ln, 1, a + 1, qij, pji, s_lb, len >= 3);
    read_msg_slot(ln, 0, lin, any);
    finalise(A, C, ln, 0, a, lin, qji, s_lb, len >= 3);
}

// One task of the hierarchy: a segment [a, b] of at least two nodes (per group;
// `active` false for groups without one) whose new sweep runs from its Lin
// (right part of its parent: type 1, forward over [a, i]) or from its Rin
// (left part: type 0, backward over [j, b]); the other message into the split
// edge is read from where an ancestor's sweep left it.  Ends with the Handshake,
// whose messages go to fmsg[j] (Lin of [j, b]) and bmsg[i] (Rin of [a, i]).
// mode 1 (the root's two halves): only the sweep, its last message stored at i
// (forward) or j (backward); mode 2 (the root's Handshake): no sweep, both
// messages into the split edge read from memory.
template <class Y, int R>
__device__ __forceinline__ void task(const Dmm16Args& A, const Ctx& C, const uint32_t* s_taps,
                                     const Lane<Y>& ln, int a, int b, int type, bool active, int mode)
{
    using M = Msg<Y::NWL>;
    using Gm = Geo<Y>;
    const int len = b - a + 1;
    const int i = a + ((len + 1) >> 1) - 1, j = i + 1;
    uint8_t* fm = reinterpret_cast<uint8_t*>(A.fmsg);
    uint8_t* bm = reinterpret_cast<uint8_t*>(A.bmsg);
    M m, inh, pij, pji;
    __syncwarp();
    if (mode == 2) {
        // the root's Handshake: both messages into the split edge from memory
        issue_msg<Y>(fm, A.fofs, C, i, ln, 0, active);
        issue_msg<Y>(bm, A.bofs, C, j, ln, 1, active);
        cp_commit();
        stage_slots<Y>(A, C, ln, active ? i : 0, active ? 2 : 0, false);
        cp_wait<0>();
        __syncwarp();
        read_msg_slot(ln, 0, inh, active);
        read_msg_slot(ln, 1, m, active);
        const Taps tp = taps_of<R>(s_taps, slot_omega(ln, 0, C, active ? i : -1));
        handshake<Y, R>(ln, 0, 1, tp, inh, m, pij, pji);
    } else {
        // the sweep's boundary message (slot 1) and, for a Handshake, the inherited
        // message at the split (slot 0), in flight with the sweep's first blocks
        issue_msg<Y>(type ? fm : bm, type ? A.fofs : A.bofs, C, type ? a : b, ln, 1, active);
        if (mode == 0) issue_msg<Y>(type ? bm : fm, type ? A.bofs : A.fofs, C, type ? j : i, ln, 0, active);
        cp_commit();
        const int count = active ? (type ? i - a : b - j) : 0;
        const int maxc = __reduce_max_sync(kFull, count);
        const int minc = __reduce_min_sync(kFull, active ? count : maxc);
        const int extra = mode == 0 ? 2 : 0;  // the Handshake's nodes follow the sweep's
        sweep<Y, R>(A, C, s_taps, ln, type ? a : b, type ? 1 : -1, count, minc, maxc, extra, 1, active, m,
                    type ? spine_fwd(a, i) : spine_bwd(j, b));
        if (mode == 1) {
            store_msg<Y>(type ? fm : bm, type ? A.fofs : A.bofs, C, type ? i : j, ln, m, active);
            return;
        }
        __syncwarp();
        // the nodes after the sweep: i then j (forward), j then i (backward); the
        // weight staged with the first of them is that of the edge (i, j)
        const int p0 = count, p1 = count + 1;
        const uint8_t* b0 = ln.ring + ((p0 / Y::KB) % RB) * Gm::BLK;
        const uint8_t* b1 = ln.ring + ((p1 / Y::KB) % RB) * Gm::BLK;
        const uint8_t* r0 = b0 + (p0 % Y::KB) * Gm::ROW;
        const uint8_t* r1 = b1 + (p1 % Y::KB) * Gm::ROW;
        const int base0 = *reinterpret_cast<const int*>(b0 + Gm::BASE_AT + 4 * (p0 % Y::KB));
        const int base1 = *reinterpret_cast<const int*>(b1 + Gm::BASE_AT + 4 * (p1 % Y::KB));
        const uint32_t ww = *reinterpret_cast<const uint32_t*>(b0 + Gm::W_AT + 4 * (p0 % Y::KB));
        const Taps tp = taps_of<R>(s_taps, active ? omega_of(ww, C, i) : 0);
        read_msg_slot(ln, 0, inh, active);
        if (type) handshake_at<Y, R>(ln, r0, base0, r1, base1, tp, m, inh, pij, pji);  // F_i swept
        else handshake_at<Y, R>(ln, r1, base1, r0, base0, tp, inh, m, pij, pji);       // B_j swept
    }
    store_msg<Y>(bm, A.bofs, C, i, ln, pji, active);
    store_msg<Y>(fm, A.fofs, C, j, ln, pij, active);
}

// ceil(n / 2^l): the longest segment at level l of the split tree of n nodes
__device__ __forceinline__ int level_max(int n, int l) { return (n + (1 << l) - 1) >> l; }

// Segment s of level `level` of the split tree of [0, n) (the left part of a
// split keeps ceil(len/2) nodes).  Returns the length (0 if an ancestor is a
// single node).
__device__ __forceinline__ int segment_of(int n, int level, int s, int& a, int& b)
{
    a = 0;
    b = n - 1;
    for (int bit = level - 1; bit >= 0; --bit) {
        const int len = b - a + 1;
        if (len <= 1) return 0;
        const int i = a + ((len + 1) >> 1) - 1;
        if ((s >> bit) & 1) a = i + 1;
        else b = i;
    }
    return b - a + 1;
}

// A group of the whole-warp layout owns the areas of its warp's groups of the
// group layout: its ring starts in the first, its message slots are those of
// the last (the ring of RB larger blocks ends before them).
template <class Y>
__device__ __forceinline__ Lane<Y> make_lane(const Dmm16Args& A, uint8_t* areas, int GD)
{
    using Ar = Area<Y::LP, typename Y::DT>;
    Lane<Y> ln;
    ln.q = (int)(threadIdx.x & 31) % Y::G;
    ln.g = (int)threadIdx.x / Y::G;
    ln.pad = ln.q * Y::LPL >= A.L;
    ln.s0 = ln.pad ? 0x5454u : 0x6160u;
    ln.s1 = ln.pad ? 0x5454u : 0x6362u;
    const int first = ln.g * (Y::G / GD), last = first + Y::G / GD - 1;
    ln.ring = areas + (size_t)first * Ar::GRP;
    ln.ms = areas + (size_t)last * Ar::GRP + RB * Ar::BLK;
    return ln;
}

__device__ __forceinline__ Ctx make_ctx(const Dmm16Args& A, int chain)
{
    Ctx C;
    C.which = A.which;
    C.H = A.H;
    C.W = A.W;
    C.L = A.L;
    C.n = A.which == 0 ? A.W : A.H;
    C.c = chain;
    C.c16 = A.cost16 != nullptr;
    C.err = A.err;
    return C;
}

// A leaf block (group layout) as a call of its own: it needs the most registers
// of the pass, and out of line it neither spills nor makes the sweeps spill.  The
// arguments are the CTA's copy of the pass arguments in shared memory and plain
// integers (a reference to the kernel parameters would force a local copy).
template <int LP, typename DT, int R>
__device__ __noinline__ void leaf_call(const Dmm16Args* A, const uint32_t* s_taps, uint8_t* areas,
                                       long long* s_lb, int chain, int a, int len, int maxlen)
{
    constexpr int GD = LP / 16;
    using YD = Lay<LP, GD, DT, KB>;
    leaf_block<YD, R>(*A, make_ctx(*A, chain), s_taps, make_lane<YD>(*A, areas, GD), a, len, maxlen, s_lb);
}

// One chain (row `chain` of the horizontal pass, column of the vertical pass)
// of Alg. Dual_MM's minorant computation by the whole CTA.
//
// Rounds, each ended by a CTA barrier: the root's two half sweeps, the root's
// Handshake, then one level per round while a level has at most one segment per
// warp (whole-warp layout) or per group (group layout); then every group walks
// the subtree of its segment depth first (group layout).  A segment is a task
// (new sweep and Handshake) if the longest segment of its level has at least 5
// nodes and a leaf block (its whole subtree at once) otherwise; the rule is the
// same for every segment of a level, so the groups that take the next level's
// segments know which ones exist.  In the depth-first part a warp decides by the
// longest segment among its own groups, which keeps its subtrees consistent
// because no other warp touches them.
//
// phase 0 runs the whole chain (every thread of the CTA).  The split pass
// splits it: phase 1 (every thread) runs the levels down to KL, one level
// further than phase 0's level-synchronous part, and stops; phase 2 (one warp)
// walks the depth-first subtrees of that warp's groups from the level-(KL+1)
// segments seg0, seg0 + 1, ... of the chain, reading everything it needs from
// memory, with no CTA barrier.
template <int LP, typename DT, int R, int NW = warps_of<LP / 16>()>
__device__ __forceinline__ void chain_g(const Dmm16Args& A, const Dmm16Args* s_args, int chain, uint8_t* smem,
                                        const uint32_t* s_taps, int phase = 0, int seg0 = 0)
{
    constexpr int GD = LP / 16;                 // lanes per group of the group layout
    constexpr bool WIDE = LP >= 64;             // a warp holds a message with >= 2 labels per lane
    using YD = Lay<LP, GD, DT, KB>;
    // the whole-warp layout stages 16 steps per block where its ring fits, else 8
    constexpr int ROOM = (32 / GD - 1) * Area<LP, DT>::GRP + RB * Area<LP, DT>::BLK;
    constexpr int KBW = RB * (16 * LP * (int)sizeof(DT) + 8 * 16) <= ROOM ? 16 : 8;
    using YW = Lay<LP, (WIDE ? 32 : GD), DT, (WIDE ? KBW : KB)>;
    // the whole-warp ring fits in front of the last area's message slots
    static_assert(!WIDE || RB * Geo<YW>::BLK <= ROOM, "whole-warp staging ring");
    using Ar = Area<LP, DT>;
    constexpr int NWARP = NW;
    constexpr int NG = NWARP * 32 / GD;         // groups per CTA
    constexpr int KL = NG >= 32 ? 5 : (NG >= 16 ? 4 : (NG >= 8 ? 3 : 2));  // log2(NG)
    static_assert((1 << KL) == NG, "groups per CTA must be a power of two");
    constexpr int NWIDE = YW::G == 32 ? NWARP : NG;  // segments one round of the wide layout takes
    uint8_t* areas = smem + 256 * tap_words<R>() * 4;
    const int gd = (int)threadIdx.x / GD, qd = (int)(threadIdx.x & 31) % GD;  // group-layout group and lane
    const Ctx C = make_ctx(A, chain);
    const int n = C.n;
    uint8_t* gtail = areas + NG * Ar::GRP;
    uint32_t* s_stk = reinterpret_cast<uint32_t*>(gtail) + gd * kStack;
    long long* s_lb = reinterpret_cast<long long*>(gtail + NG * kStack * 4) + gd;
    if (qd == 0) *s_lb = 0;
    const int warp = (int)threadIdx.x >> 5;
    int round = 0;   // 0, 1: the root; then level = round - 1
    bool dfs = false;
    int sp = 0;      // depth-first stack size (warp-uniform)
    // the first level walked depth first: KL, or KL + 1 in the split pass
    const int LD = phase == 0 ? KL : KL + 1;
    if (phase != 2) {
        // zero boundary messages at both chain ends
        if (threadIdx.x < 32) {
            const Lane<YW> lw = make_lane<YW>(A, areas, GD);
            Msg<YW::NWL> zero;
            zero_msg(zero);
            store_msg<YW>(reinterpret_cast<uint8_t*>(A.fmsg), A.fofs, C, 0, lw, zero, lw.g == 0);
            store_msg<YW>(reinterpret_cast<uint8_t*>(A.bmsg), A.bofs, C, n - 1, lw, zero, lw.g == 0);
        }
        __syncthreads();
    } else {
        // this warp's groups take the level-LD segments seg0 + (their index in the warp)
        dfs = true;
        const int s = seg0 + gd % (32 / GD);
        int a = 0, b = 0;
        const int l = segment_of(n, LD, s, a, b);
        if (qd == 0)
            s_stk[0] = (uint32_t)(l > 0 ? a : 0) | ((uint32_t)(l > 0 ? b : 0) << 15) |
                       ((uint32_t)(s & 1) << 30) | (l > 0 ? 0x80000000u : 0u);
        sp = 1;
        __syncwarp();
    }
    int rounds = 0;  // bounded: at most KL + 2 level rounds and 2n depth-first steps
#pragma unroll 1
    for (;;) {
        if (++rounds > 4 * n + 64 || sp > kStack - 2) {  // cannot happen: report it rather than spin
            if (qd == 0) atomicOr(C.err, kDevErrIndex);
            break;
        }
        // ---- this round's work: 0 nothing, 1 task (wide layout), 2 task (group
        // layout), 3 leaf block (group layout)
        int kind = 0, a = 0, b = 0, type = 0, len = 0, maxlen = 0, mode = 0;
        if (!dfs) {
            const int level = round < 2 ? 0 : round - 1;
            if (n <= 4) {
                if (warp == 0) {
                    kind = 3;
                    len = gd == 0 ? n : 0;
                    maxlen = n;
                }
            } else if (round < 2) {
                // the root: its two halves (mode 1), then its Handshake (mode 2)
                if (round == 0 && YW::G == 32 ? warp < 2 : warp == 0) {
                    const int me = YW::G == 32 ? warp : gd;
                    kind = 1;
                    mode = round == 0 ? 1 : 2;
                    len = round == 0 ? (me < 2 ? n : 0) : (me == 0 ? n : 0);
                    b = len > 0 ? n - 1 : 0;
                    type = me == 0 ? 1 : 0;  // forward half, backward half
                }
            } else if (level < LD && level_max(n, level - 1) >= 5) {
                const int nseg = 1 << level;
                if (nseg <= NWIDE && level_max(n, level) >= 5) {
                    // whole-warp layout (or the group layout when LP < 64)
                    const int s = YW::G == 32 ? warp : gd;
                    if ((YW::G == 32 ? warp : warp * (32 / YW::G)) < nseg) {
                        len = s < nseg ? segment_of(n, level, s, a, b) : 0;
                        if (len == 0) a = b = 0;
                        type = s & 1;
                        kind = 1;
                    }
                } else if (warp * (32 / GD) < nseg) {
                    len = gd < nseg ? segment_of(n, level, gd, a, b) : 0;
                    if (len == 0) a = b = 0;
                    type = gd & 1;
                    kind = level_max(n, level) >= 5 ? 2 : 3;
                    maxlen = __reduce_max_sync(kFull, len);
                }
            } else {
                // from level KL on every group walks its segment's subtree depth
                // first (in the split pass, from level KL + 1, in phase 2)
                if (phase == 1) break;
                dfs = true;
                if (level == KL && level_max(n, KL - 1) >= 5) {
                    const int l = segment_of(n, KL, gd, a, b);
                    // entry: a | b << 15 | type << 30 | valid << 31 (chains of at most 32768 nodes)
                    if (qd == 0)
                        s_stk[0] = (uint32_t)(l > 0 ? a : 0) | ((uint32_t)(l > 0 ? b : 0) << 15) |
                                   ((uint32_t)(gd & 1) << 30) | (l > 0 ? 0x80000000u : 0u);
                    sp = 1;
                }
                __syncwarp();
                continue;
            }
        } else {
            if (sp == 0) break;
            --sp;
            const uint32_t e = s_stk[sp];
            __syncwarp();
            a = (int)(e & 0x7fffu);
            b = (int)((e >> 15) & 0x7fffu);
            type = (int)((e >> 30) & 1u);
            len = (e >> 31) ? b - a + 1 : 0;
            maxlen = __reduce_max_sync(kFull, len);
            kind = maxlen >= 5 ? 2 : (maxlen >= 1 ? 3 : 0);
        }
        if (kind == 1) {
            task<YW, R>(A, C, s_taps, make_lane<YW>(A, areas, GD), a, b, type, len >= 2, mode);
        } else if (kind == 2) {
            task<YD, R>(A, C, s_taps, make_lane<YD>(A, areas, GD), a, b, type, len >= 2, 0);
            if (dfs) {
                const int i = a + ((len + 1) >> 1) - 1, j = i + 1;
                if (qd == 0) {
                    // right part, then the left part on top (visited first)
                    const uint32_t v = len >= 2 ? 0x80000000u : 0u;
                    s_stk[sp] = (uint32_t)j | ((uint32_t)b << 15) | (1u << 30) | v;
                    s_stk[sp + 1] = (uint32_t)a | ((uint32_t)i << 15) | v;
                }
                sp += 2;
                __syncwarp();
            }
        } else if (kind == 3) {
            leaf_call<LP, DT, R>(s_args, s_taps, areas, s_lb, chain, a, len, maxlen);
        }
        if (!dfs) {
            __syncthreads();
            if (n <= 4) break;
            ++round;
        }
    }
    if (A.lb != nullptr && qd == 0 && *s_lb != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(A.lb), (unsigned long long)*s_lb);
}

template <int LP, int R, typename DT, int NW = warps_of<LP / 16>()>
constexpr int smem_g()
{
    constexpr int NG = NW * 32 / (LP / 16);
    return 256 * tap_words<R>() * 4 + NG * (Area<LP, DT>::GRP + kStack * 4 + 8) +
           (int)((sizeof(Dmm16Args) + 15) & ~(size_t)15);
}

// Launched with programmatic stream serialisation: the taps table (which no
// pass writes) is staged while the previous pass drains; everything else waits
// for that grid (griddepcontrol.wait).  Without the attribute both are no-ops.
template <int LP, int R, typename DT, int NW = warps_of<LP / 16>(), int PH = 0>
__global__ void __launch_bounds__(NW * 32, 24 / NW) dmg_kernel(const Dmm16Args A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* s_taps = reinterpret_cast<uint32_t*>(smem);
    constexpr int TW = tap_words<R>();
    for (int t = threadIdx.x; t < 256 * TW; t += blockDim.x) s_taps[t] = A.taps16[(t / TW) * kTapW + t % TW];
    // the arguments, for the leaf blocks' calls, at the end of the dynamic shared memory
    Dmm16Args* s_args = reinterpret_cast<Dmm16Args*>(smem + smem_g<LP, R, DT, NW>() -
                                                     ((sizeof(Dmm16Args) + 15) & ~(size_t)15));
    if (threadIdx.x == 0) *s_args = A;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();
    chain_g<LP, DT, R, NW>(A, s_args, blockIdx.x, smem, s_taps, PH);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Persistent form over the chains of many pairs of one label class (the
// batched solve): every CTA takes (pair, chain) tasks from a work counter,
// longest chains first, until none are left.  All pairs share the penalty (one
// taps table).  A chain's work is chain_g's, exactly as in dmg_kernel.
template <int LP, int R, typename DT>
__global__ void __launch_bounds__(warps_of<LP / 16>() * 32, 24 / warps_of<LP / 16>())
    dmg_batch_kernel(const __grid_constant__ Batch16Args B)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_t;
    uint32_t* s_taps = reinterpret_cast<uint32_t*>(smem);
    constexpr int TW = tap_words<R>();
    const uint32_t* taps = B.descs[0].taps16;
    for (int t = threadIdx.x; t < 256 * TW; t += blockDim.x) s_taps[t] = taps[(t / TW) * kTapW + t % TW];
    Dmm16Args* s_args = reinterpret_cast<Dmm16Args*>(smem + smem_g<LP, R, DT>() -
                                                     ((sizeof(Dmm16Args) + 15) & ~(size_t)15));
#pragma unroll 1
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(B.counter, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= B.n_tasks) break;
        const int2 tk = B.tasks[t];
        if (threadIdx.x == 0) *s_args = B.descs[tk.x];
        __syncthreads();
        chain_g<LP, DT, R>(B.descs[tk.x], s_args, tk.y, smem, s_taps);
        __syncthreads();
    }
}

// The split pass, for chains whose depth-first part would leave some SMs
// idle: dmg_kernel<..., 1> runs every chain's levels down to KL (chain_g phase
// 1, one CTA per chain), then this kernel (launched after it; its
// griddepcontrol.wait waits for that grid and its memory) shares the
// depth-first part, cut into 2 NW units per chain (the level-(KL+1) segments of
// one warp's groups each), among persistent CTAs: every warp takes units from
// one counter (pool[0]) until none is left.  The last CTA out zeroes the
// counters (pool[0], pool[1]) for the next launch.  Results equal dmg_kernel's
// bit for bit.
template <int LP, int R, typename DT, int NW = warps_of<LP / 16>()>
__global__ void __launch_bounds__(NW * 32, 24 / NW) dmg_units_kernel(const Dmm16Args A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_last;
    constexpr int GD = LP / 16, GPW = 32 / GD, NU = 2 * NW;
    uint32_t* s_taps = reinterpret_cast<uint32_t*>(smem);
    constexpr int TW = tap_words<R>();
    for (int t = threadIdx.x; t < 256 * TW; t += blockDim.x) s_taps[t] = A.taps16[(t / TW) * kTapW + t % TW];
    Dmm16Args* s_args = reinterpret_cast<Dmm16Args*>(smem + smem_g<LP, R, DT, NW>() -
                                                     ((sizeof(Dmm16Args) + 15) & ~(size_t)15));
    if (threadIdx.x == 0) *s_args = A;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();
    int* const P = A.pool;
    const int chains = A.which == 0 ? A.H : A.W;
    const int units = chains * NU;
    const int lane = (int)threadIdx.x & 31;
#pragma unroll 1
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(P, 1);
        u = __shfl_sync(kFull, u, 0);
        if (u >= units) break;
        chain_g<LP, DT, R, NW>(A, s_args, u / NU, smem, s_taps, 2, (u % NU) * GPW);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(P + 1, 1) == (int)gridDim.x - 1;
        if (s_last) {
            P[0] = 0;
            __threadfence();
            P[1] = 0;
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

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

template <int LP, int R, typename DT, int NW = warps_of<LP / 16>()>
cudaError_t launch_one(const Dmm16Args& a, cudaStream_t s)
{
    const int smem = smem_g<LP, R, DT, NW>();
    static std::atomic<int> done[kMaxDevices];
    const cudaError_t e = ensure_smem(dmg_kernel<LP, R, DT, NW>, smem, done);
    if (e != cudaSuccess) return e;
    const int chains = a.which == 0 ? a.H : a.W;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(chains);
    cfg.blockDim = dim3(NW * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, dmg_kernel<LP, R, DT, NW>, a);
}

// the split pass: the levels down to KL with one CTA per chain, then the
// depth-first units on as many persistent CTAs as fit at once
template <int LP, int R, typename DT, int NW = warps_of<LP / 16>()>
cudaError_t launch_split(const Dmm16Args& a, cudaStream_t s)
{
    const int smem = smem_g<LP, R, DT, NW>();
    static std::atomic<int> done_t[kMaxDevices], done_u[kMaxDevices];
    cudaError_t e = ensure_smem(dmg_kernel<LP, R, DT, NW, 1>, smem, done_t);
    if (e == cudaSuccess) e = ensure_smem(dmg_units_kernel<LP, R, DT, NW>, smem, done_u);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dmg_units_kernel<LP, R, DT, NW>,
                                                          NW * 32, smem);
    if (e != cudaSuccess) return e;
    const int chains = a.which == 0 ? a.H : a.W;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NW * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(chains);
    e = cudaLaunchKernelEx(&cfg, dmg_kernel<LP, R, DT, NW, 1>, a);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(std::max(1, std::min(chains * 2 * NW, sms * per_sm)));
    return cudaLaunchKernelEx(&cfg, dmg_units_kernel<LP, R, DT, NW>, a);
}

// one pass: split when a.pool is set (and the chains have units), else one
// CTA per chain.  Measured at 1242x375x128: the horizontal pass (375 chains for
// 456 CTA slots) takes 0.448 ms split against 0.467 ms; the vertical pass gains
// nothing (0.384 ms either way) and stays one CTA per chain; units cut at level
// KL rather than KL + 1 made the horizontal pass slower (0.483 ms).
template <int LP, int R, typename DT, int NW = warps_of<LP / 16>()>
cudaError_t launch_pass(const Dmm16Args& a, cudaStream_t s)
{
    constexpr int NG = NW * (32 / (LP / 16));
    constexpr int KL = NG >= 32 ? 5 : (NG >= 16 ? 4 : (NG >= 8 ? 3 : 2));
    const int n = a.which == 0 ? a.W : a.H;
    const bool units = n > 4 && ((n + (1 << KL) - 1) >> KL) >= 5;
    return a.pool != nullptr && units ? launch_split<LP, R, DT, NW>(a, s)
                                      : launch_one<LP, R, DT, NW>(a, s);
}

template <int LP, int R, typename DT>
cudaError_t launch_batch_one(const Batch16Args& b, cudaStream_t s)
{
    const int smem = smem_g<LP, R, DT>();
    static std::atomic<int> done[kMaxDevices];
    const cudaError_t e = ensure_smem(dmg_batch_kernel<LP, R, DT>, smem, done);
    if (e != cudaSuccess) return e;
    dmg_batch_kernel<LP, R, DT><<<b.grid, warps_of<LP / 16>() * 32, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace kg

// Launcher of one label class (G lanes of 16 labels per group in the group
// layout); each is instantiated in its own translation unit.
// The vertical pass at 128 labels (1242 chains of 375 nodes on the benchmark
// frame) runs CTAs of 4 warps: five fit on an SM, so the chains take 1.6 waves
// instead of 2.7, and more top levels (latency-bound) overlap per SM.  Measured
// per pass at 1242x375x128: 0.399 ms with 4 warps against 0.425 (8) and 0.432
// (2); the horizontal pass is fastest with 8.
template <int G, typename DT>
cudaError_t launch_g(const Dmm16Args& a, int radius, cudaStream_t s)
{
    if constexpr (G == 8) {
        if (a.which == 1) {
            switch (radius) {
                case 1: return kg::launch_one<16 * G, 1, DT, 4>(a, s);
                case 2: return kg::launch_one<16 * G, 2, DT, 4>(a, s);
                default: return kg::launch_one<16 * G, 4, DT, 4>(a, s);
            }
        }
    }
    // the split pass from 128 labels on (at 64 labels, the two concurrent layers
    // of optical flow lost 3 % to it)
    if constexpr (G >= 8) {
        switch (radius) {
            case 1: return kg::launch_pass<16 * G, 1, DT>(a, s);
            case 2: return kg::launch_pass<16 * G, 2, DT>(a, s);
            default: return kg::launch_pass<16 * G, 4, DT>(a, s);
        }
    }
    switch (radius) {
        case 1: return kg::launch_one<16 * G, 1, DT>(a, s);
        case 2: return kg::launch_one<16 * G, 2, DT>(a, s);
        default: return kg::launch_one<16 * G, 4, DT>(a, s);
    }
}

template <int G, typename DT>
cudaError_t launch_g_batch(const Batch16Args& b, int radius, cudaStream_t s)
{
    switch (radius) {
        case 1: return kg::launch_batch_one<16 * G, 1, DT>(b, s);
        case 2: return kg::launch_batch_one<16 * G, 2, DT>(b, s);
        default: return kg::launch_batch_one<16 * G, 4, DT>(b, s);
    }
}

}  // namespace dm
