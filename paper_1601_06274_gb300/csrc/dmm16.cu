// Dual MM pass with packed 16-bit message arithmetic (the fast path).
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

#include "dm_internal.cuh"

namespace dm {
namespace {

constexpr int kWarps = 8;
constexpr int kPF = 4;  // prefetch depth of a sweep
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
    __device__ __forceinline__ size_t pix(int k) const
    {
        return which == 0 ? (size_t)c * W + k : (size_t)k * W + c;
    }
};

// raw unary data of one node for this lane
template <int NP, typename DT>
struct Raw {
    uint32_t d[(NP * 2 * sizeof(DT) + 3) / 4];  // deltas of lambda_in
    uint32_t c[(NP * 2 + 3) / 4];                // cost bytes (horizontal pass)
    int base;                                    // base of lambda_in
    int om;                                      // omega of the edge used at this step
};

template <int NP, typename DT>
__device__ __forceinline__ void load_raw(const Dmm16Args& A, const Ctx16& C, int k, int edge,
                                         int lane, bool pad, Raw<NP, DT>& r)
{
    const size_t pix = C.pix(k);
    r.base = __ldg(A.base_in + pix);
    r.om = edge >= 0 ? (int)__ldg(A.wedge + C.pix(edge)) : 0;
    if (pad) return;
    const size_t e0 = pix * (size_t)C.L + (size_t)lane * 2 * NP;
    const DT* dp = reinterpret_cast<const DT*>(A.delta_in) + e0;
    if constexpr (sizeof(DT) == 1) {
        if constexpr (NP == 1) r.d[0] = __ldg(reinterpret_cast<const uint16_t*>(dp));
        else if constexpr (NP == 2) r.d[0] = __ldg(reinterpret_cast<const uint32_t*>(dp));
        else { const uint2 v = __ldg(reinterpret_cast<const uint2*>(dp)); r.d[0] = v.x; r.d[1] = v.y; }
    } else {
        if constexpr (NP == 1) r.d[0] = __ldg(reinterpret_cast<const uint32_t*>(dp));
        else if constexpr (NP == 2) { const uint2 v = __ldg(reinterpret_cast<const uint2*>(dp)); r.d[0] = v.x; r.d[1] = v.y; }
        else { const uint4 v = __ldg(reinterpret_cast<const uint4*>(dp)); r.d[0] = v.x; r.d[1] = v.y; r.d[2] = v.z; r.d[3] = v.w; }
    }
    if (C.which == 0) {
        const uint8_t* cp = A.cost + e0;
        if constexpr (NP == 1) r.c[0] = __ldg(reinterpret_cast<const uint16_t*>(cp));
        else if constexpr (NP == 2) r.c[0] = __ldg(reinterpret_cast<const uint32_t*>(cp));
        else { const uint2 v = __ldg(reinterpret_cast<const uint2*>(cp)); r.c[0] = v.x; r.c[1] = v.y; }
    }
}

// byte pairs (b[2p], b[2p+1]) of a little-endian byte vector -> zero-extended 16-bit pairs
template <int NP>
__device__ __forceinline__ uint32_t unpack_u8(const uint32_t* w, int p)
{
    const uint32_t word = w[p >> 1];
    return (p & 1) ? __byte_perm(word, 0, 0x4342) : __byte_perm(word, 0, 0x4140);
}

// packed unary theta' (vector part) and the cost part alone
template <int NP, typename DT>
__device__ __forceinline__ void assemble(const Raw<NP, DT>& r, int which, bool pad,
                                         uint32_t (&th)[NP], uint32_t (&cv)[NP])
{
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint32_t d;
        if constexpr (sizeof(DT) == 1) d = unpack_u8<NP>(r.d, p);
        else d = r.d[p];
        const uint32_t c = (which == 0) ? unpack_u8<NP>(r.c, p) : 0u;
        cv[p] = c;
        th[p] = pad ? kInf2 : vadd2(d, c);
    }
}

__device__ __forceinline__ Taps taps_of(const uint32_t* s_taps, int om)
{
    const uint4 v = *reinterpret_cast<const uint4*>(s_taps + om * kTapW);
    Taps t;
    t.t[0] = v.x; t.t[1] = v.y; t.t[2] = v.z; t.t[3] = v.w;
    t.p2 = (int)s_taps[om * kTapW + kTapP2];
    return t;
}

template <int NP>
__device__ __forceinline__ void store_msg(const Dmm16Args& A, uint32_t* buf, int* ofs,
                                          const Ctx16& C, int pos, int lane,
                                          const uint32_t (&m)[NP], int off)
{
    uint32_t* p = buf + ((size_t)C.c * C.n + pos) * C.KP2 + lane * NP;
    if constexpr (NP == 1) p[0] = m[0];
    else if constexpr (NP == 2) *reinterpret_cast<uint2*>(p) = make_uint2(m[0], m[1]);
    else *reinterpret_cast<uint4*>(p) = make_uint4(m[0], m[1], m[2], m[3]);
    if (lane == 0) ofs[(size_t)C.c * C.n + pos] = off;
}

template <int NP>
__device__ __forceinline__ void load_msg(const uint32_t* buf, const int* ofs, const Ctx16& C,
                                         int pos, int lane, uint32_t (&m)[NP], int& off)
{
    const uint32_t* p = buf + ((size_t)C.c * C.n + pos) * C.KP2 + lane * NP;
    if constexpr (NP == 1) m[0] = p[0];
    else if constexpr (NP == 2) { const uint2 v = *reinterpret_cast<const uint2*>(p); m[0] = v.x; m[1] = v.y; }
    else { const uint4 v = *reinterpret_cast<const uint4*>(p); m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w; }
    off = ofs[(size_t)C.c * C.n + pos];
}

// Output of a node that is a single node of the hierarchy: it keeps theta +
// Lin + Rin.  lambda_out = cost + Lin + Rin (horizontal) or Lin + Rin
// (vertical); the vertical pass can also emit the label and the node's share
// of the lower bound (min over labels of lambda_h + lambda_v).
template <int NP, typename DT>
__device__ __forceinline__ void finalise(const Dmm16Args& A, const Ctx16& C, int k, int lane,
                                         bool pad, const uint32_t (&th)[NP], int th_base,
                                         const uint32_t (&cv)[NP], const uint32_t (&lin)[NP],
                                         int lin_off, const uint32_t (&rin)[NP], int rin_off,
                                         long long& lb_acc)
{
    const size_t pix = C.pix(k);
    uint32_t v[NP];
    uint32_t bad = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        v[p] = vadd2(vadd2(lin[p], rin[p]), C.which == 0 ? cv[p] : 0u);
        bad |= v[p];
    }
    if (lane == 0) A.base_out[pix] = lin_off + rin_off;
    if (!pad) {
        if constexpr (sizeof(DT) == 1) {
            // every delta is in [0, 255]: the host only picks 8-bit storage when it must be
            if (bad & 0xff00ff00u) atomicOr(A.err, kDevErrRange);
            uint8_t* dp = reinterpret_cast<uint8_t*>(A.delta_out) + pix * (size_t)C.L + lane * 2 * NP;
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
                                                       pix * (size_t)C.L + lane * 2 * NP);
            if constexpr (NP == 1) dp[0] = v[0];
            else if constexpr (NP == 2) *reinterpret_cast<uint2*>(dp) = make_uint2(v[0], v[1]);
            else *reinterpret_cast<uint4*>(dp) = make_uint4(v[0], v[1], v[2], v[3]);
        }
    }
    if (A.labels != nullptr || A.lb != nullptr) {
        // nu = lambda_h + lambda_v = theta + Lin + Rin (vertical pass: theta = lambda_h)
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

// Segment s of level `level` of the split tree of [0, n) (left part ceil(len/2)).
__device__ __forceinline__ bool segment16(int n, int level, int s, int& a, int& b)
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

// One sweep of `count` Msg steps.  dir = +1: forward from node k0 (messages
// enter k0+1, k0+2, ...; edge of step k is k).  dir = -1: backward from k0
// (messages enter k0-1, ...; edge of step k is k-1).  `msg`/`off` hold the
// boundary message on entry and the last message on exit.  Messages entering
// the positions listed in save[0..nsave) (in visiting order) are stored.
template <int NP, int R, bool PAD, typename DT>
__device__ __forceinline__ void sweep16(const Dmm16Args& A, const Ctx16& C, const uint32_t* s_taps,
                                        int k0, int dir, int count, uint32_t (&msg)[NP], int& off,
                                        const int* save, int nsave, uint32_t* sbuf, int* sofs,
                                        int lane, bool pad)
{
    if (count <= 0) return;
    Raw<NP, DT> ring[kPF];
#pragma unroll
    for (int u = 0; u < kPF; ++u)
        if (u < count) {
            const int k = k0 + dir * u;
            load_raw<NP, DT>(A, C, k, dir > 0 ? k : k - 1, lane, pad, ring[u]);
        }
    int si = 0;
    int next = nsave > 0 ? save[0] : -1;
    for (int s = 0; s < count; s += kPF) {
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            if (s + u < count) {
                const int k = k0 + dir * (s + u);
                uint32_t th[NP], cv[NP], x[NP];
                assemble<NP, DT>(ring[u], C.which, pad, th, cv);
                const Taps tp = taps_of(s_taps, ring[u].om);
                off += ring[u].base;
#pragma unroll
                for (int p = 0; p < NP; ++p) x[p] = vadd2(th[p], msg[p]);
                if (s + u + kPF < count) {
                    const int kn = k + dir * kPF;
                    load_raw<NP, DT>(A, C, kn, dir > 0 ? kn : kn - 1, lane, pad, ring[u]);
                }
                msg16<NP, R, PAD>(x, msg, off, tp, lane, pad);
                const int pos = k + dir;
                if (pos == next) {
                    store_msg<NP>(A, sbuf, sofs, C, pos, lane, msg, off);
                    ++si;
                    next = si < nsave ? save[si] : -1;
                }
            }
        }
    }
}

// The split points whose inherited message a fresh sweep must leave behind.
// Forward sweep of a segment with left part [a, i]: the split points of [a, i],
// of its left part, and so on (offsets (i-a) >> t from a), visited in
// increasing order.  Backward sweep with right part [j, b]: the first nodes of
// the right parts of [j, b], of its right part, and so on, visited in
// decreasing order.  Returns the count (<= 20).
__device__ __forceinline__ int spine_fwd(int a, int i, int* out)
{
    int cnt = 0, tmp[20];
    for (int o = (i - a) >> 1; o > 0; o >>= 1) tmp[cnt++] = a + o;  // decreasing
    for (int t = 0; t < cnt; ++t) out[t] = tmp[cnt - 1 - t];
    return cnt;
}

__device__ __forceinline__ int spine_bwd(int j, int b, int* out)
{
    int cnt = 0, tmp[20];
    int s = j;
    while (b - s + 1 >= 3) {
        s = s + ((b - s + 2) >> 1);  // first node of the right part of [s, b]
        if (s < b) tmp[cnt++] = s;
    }
    // tmp is increasing; the backward sweep visits decreasing positions
    for (int t = 0; t < cnt; ++t) out[t] = tmp[cnt - 1 - t];
    return cnt;
}

template <int NP, int R, bool PAD, typename DT>
__device__ __forceinline__ void handshake16(const Dmm16Args& A, const Ctx16& C,
                                            const uint32_t* s_taps, int a, int b, int i, int j,
                                            const uint32_t (&Fi)[NP], int offF,
                                            const uint32_t (&Bj)[NP], int offB, int lane,
                                            bool pad, long long& lb_acc)
{
    Raw<NP, DT> ri, rj;
    load_raw<NP, DT>(A, C, i, i, lane, pad, ri);
    load_raw<NP, DT>(A, C, j, -1, lane, pad, rj);
    uint32_t thi[NP], cvi[NP], thj[NP], cvj[NP];
    assemble<NP, DT>(ri, C.which, pad, thi, cvi);
    assemble<NP, DT>(rj, C.which, pad, thj, cvj);
    const Taps tp = taps_of(s_taps, ri.om);
    uint32_t x[NP], phi_ji[NP], phi_ij[NP];
    // message j -> i
    int o_ji = offB + rj.base;
#pragma unroll
    for (int p = 0; p < NP; ++p) x[p] = vadd2(thj[p], Bj[p]);
    msg16<NP, R, PAD>(x, phi_ji, o_ji, tp, lane, pad);
    // half of the total min-marginal at i, shared to the right: floor(m_i / 2) - phi_ji
    const int o_m = offF + ri.base + o_ji;  // even
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const uint32_t mi = vadd2(vadd2(Fi[p], thi[p]), phi_ji[p]);  // >= 0 in both halves
        x[p] = vsub2((mi >> 1) & 0x7fff7fffu, phi_ji[p]);
    }
    int o_ij = (o_m >> 1) - o_ji;
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
    int o_b = -o_ij;
    msg16<NP, R, true>(x, phi_ji, o_b, tp, lane, pad);
    // left child [a, i] gets Rin = phi_ji; right child [j, b] gets Lin = phi_ij
    if (i == a)
        finalise<NP, DT>(A, C, i, lane, pad, thi, ri.base, cvi, Fi, offF, phi_ji, o_b, lb_acc);
    else
        store_msg<NP>(A, A.bmsg, A.bofs, C, i, lane, phi_ji, o_b);
    if (j == b)
        finalise<NP, DT>(A, C, j, lane, pad, thj, rj.base, cvj, phi_ij, o_ij, Bj, offB, lb_acc);
    else
        store_msg<NP>(A, A.fmsg, A.fofs, C, j, lane, phi_ij, o_ij);
}

template <int NP, int R, bool PAD, typename DT>
__global__ void __launch_bounds__(kWarps * 32, 3) dmm16_kernel(const Dmm16Args A)
{
    __shared__ __align__(16) uint32_t s_taps[256 * kTapW];
    for (int t = threadIdx.x; t < 256 * kTapW; t += blockDim.x) s_taps[t] = A.taps16[t];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Ctx16 C;
    C.which = A.which;
    C.H = A.H;
    C.W = A.W;
    C.L = A.L;
    C.n = A.which == 0 ? A.W : A.H;
    C.c = blockIdx.x;
    C.KP2 = 32 * NP;
    const int n = C.n;
    const bool pad = PAD && (lane * 2 * NP >= A.L);
    long long lb_acc = 0;
    uint32_t zero[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) zero[p] = 0u;
    // zero boundary messages at both chain ends
    if (warp == 0) {
        store_msg<NP>(A, A.fmsg, A.fofs, C, 0, lane, zero, 0);
        store_msg<NP>(A, A.bmsg, A.bofs, C, n - 1, lane, zero, 0);
    }
    __syncthreads();

    if (n == 1) {
        if (warp == 0) {
            Raw<NP, DT> r;
            load_raw<NP, DT>(A, C, 0, -1, lane, pad, r);
            uint32_t th[NP], cv[NP];
            assemble<NP, DT>(r, C.which, pad, th, cv);
            finalise<NP, DT>(A, C, 0, lane, pad, th, r.base, cv, zero, 0, zero, 0, lb_acc);
        }
    } else {
        int levels = 0;
        while ((1 << levels) < n) ++levels;
        int save[20];
        // ---- level 0: both halves swept in parallel, then the root Handshake
        {
            const int a = 0, b = n - 1;
            const int i = ((n + 1) >> 1) - 1, j = i + 1;
            uint32_t m[NP];
            int off = 0;
#pragma unroll
            for (int p = 0; p < NP; ++p) m[p] = 0u;
            if (warp == 0) {
                const int ns = spine_fwd(a, i, save);
                sweep16<NP, R, PAD, DT>(A, C, s_taps, a, +1, i - a, m, off, save, ns, A.fmsg,
                                        A.fofs, lane, pad);
                store_msg<NP>(A, A.fmsg, A.fofs, C, i, lane, m, off);
            } else if (warp == 1) {
                const int ns = spine_bwd(j, b, save);
                sweep16<NP, R, PAD, DT>(A, C, s_taps, b, -1, b - j, m, off, save, ns, A.bmsg,
                                        A.bofs, lane, pad);
                store_msg<NP>(A, A.bmsg, A.bofs, C, j, lane, m, off);
            }
            __syncthreads();
            if (warp == 0) {
                uint32_t Fi[NP], Bj[NP];
                int oF, oB;
                load_msg<NP>(A.fmsg, A.fofs, C, i, lane, Fi, oF);
                load_msg<NP>(A.bmsg, A.bofs, C, j, lane, Bj, oB);
                handshake16<NP, R, PAD, DT>(A, C, s_taps, a, b, i, j, Fi, oF, Bj, oB, lane, pad,
                                            lb_acc);
            }
            __syncthreads();
        }
        // ---- levels >= 1: one warp per segment, sweep + Handshake
        for (int level = 1; level < levels; ++level) {
            const int nseg = 1 << level;
            for (int s = warp; s < nseg; s += kWarps) {
                int a, b;
                if (!segment16(n, level, s, a, b) || b <= a) continue;
                const int i = a + ((b - a + 2) >> 1) - 1, j = i + 1;
                uint32_t Fi[NP], Bj[NP];
                int oF, oB;
                if (s & 1) {
                    // right child: Lin changed, left messages recomputed from a
                    load_msg<NP>(A.fmsg, A.fofs, C, a, lane, Fi, oF);
                    const int ns = spine_fwd(a, i, save);
                    sweep16<NP, R, PAD, DT>(A, C, s_taps, a, +1, i - a, Fi, oF, save, ns, A.fmsg,
                                            A.fofs, lane, pad);
                    load_msg<NP>(A.bmsg, A.bofs, C, j, lane, Bj, oB);
                } else {
                    // left child: Rin changed, right messages recomputed from b
                    load_msg<NP>(A.bmsg, A.bofs, C, b, lane, Bj, oB);
                    const int ns = spine_bwd(j, b, save);
                    sweep16<NP, R, PAD, DT>(A, C, s_taps, b, -1, b - j, Bj, oB, save, ns, A.bmsg,
                                            A.bofs, lane, pad);
                    load_msg<NP>(A.fmsg, A.fofs, C, i, lane, Fi, oF);
                }
                handshake16<NP, R, PAD, DT>(A, C, s_taps, a, b, i, j, Fi, oF, Bj, oB, lane, pad,
                                            lb_acc);
            }
            __syncthreads();
        }
    }
    if (A.lb != nullptr && lane == 0 && lb_acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(A.lb), (unsigned long long)lb_acc);
}

template <int NP, int R, typename DT>
cudaError_t launch_nrd(const Dmm16Args& a, cudaStream_t s)
{
    const int chains = a.which == 0 ? a.H : a.W;
    if (a.L == 32 * 2 * NP)
        dmm16_kernel<NP, R, false, DT><<<chains, kWarps * 32, 0, s>>>(a);
    else
        dmm16_kernel<NP, R, true, DT><<<chains, kWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NP, typename DT>
cudaError_t launch_nd(const Dmm16Args& a, int radius, cudaStream_t s)
{
    switch (radius) {
        case 1: return launch_nrd<NP, 1, DT>(a, s);
        case 2: return launch_nrd<NP, 2, DT>(a, s);
        default: return launch_nrd<NP, 4, DT>(a, s);
    }
}

template <typename DT>
cudaError_t launch_d(const Dmm16Args& a, int np, int radius, cudaStream_t s)
{
    switch (np) {
        case 1: return launch_nd<1, DT>(a, radius, s);
        case 2: return launch_nd<2, DT>(a, radius, s);
        default: return launch_nd<4, DT>(a, radius, s);
    }
}

__global__ void validate_edges_kernel(const uint8_t* __restrict__ wh, const uint8_t* __restrict__ wv,
                                      int H, int W, const int32_t* __restrict__ taps,
                                      int32_t* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * W) return;
    const int x = i % W, y = i / W;
    bool bad = false;
    if (x + 1 < W) bad |= taps[(int)wh[i] * kTapW + kTapValid] == 0;
    if (y + 1 < H) bad |= taps[(int)wv[i] * kTapW + kTapValid] == 0;
    if (bad) atomicOr(err, kDevErrBadOmega);
}

__global__ void duals_to_i32_kernel(const int32_t* __restrict__ base, const void* __restrict__ delta,
                                    int delta_bytes, long long n_px, int L, int32_t* __restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_px * L) return;
    const long long px = t / L;
    const int d = delta_bytes == 1 ? (int)static_cast<const uint8_t*>(delta)[t]
                                   : (int)static_cast<const int16_t*>(delta)[t];
    out[t] = base[px] + d;
}

}  // namespace

cudaError_t launch_dmm16_pass(const Dmm16Args& a, int np, int radius, int delta_bytes,
                              cudaStream_t s)
{
    if (delta_bytes == 1) return launch_d<uint8_t>(a, np, radius, s);
    return launch_d<int16_t>(a, np, radius, s);
}

cudaError_t launch_validate_edges(const uint8_t* wh, const uint8_t* wv, int H, int W,
                                  const int32_t* taps, int32_t* err, cudaStream_t s)
{
    const int n = H * W;
    validate_edges_kernel<<<(n + 255) / 256, 256, 0, s>>>(wh, wv, H, W, taps, err);
    return cudaGetLastError();
}

cudaError_t launch_duals_to_i32(const int32_t* base, const void* delta, int delta_bytes,
                                long long n_px, int L, int32_t* out, cudaStream_t s)
{
    const long long total = n_px * L;
    duals_to_i32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(base, delta, delta_bytes,
                                                                          n_px, L, out);
    return cudaGetLastError();
}

}  // namespace dm
