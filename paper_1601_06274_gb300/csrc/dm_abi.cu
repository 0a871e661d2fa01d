// C ABI of libdm.so (declared in include/dm.h): context, workspace layout,
// argument checking and the launch sequence of the stereo hot path of
// arXiv 1601.06274 (cost volume -> Dual MM -> primal-dual refinement).

#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dm_internal.cuh"

#include "dm_ctx.cuh"

namespace {

constexpr int kMaxIters = 4096;
constexpr int kMaxDelta16 = 255 + 2 * (8000 + 1);  // largest delta the 16-bit kernel admits
// the lane-group kernel: deltas up to 8000 keep its padded labels (read as
// 16383) out of every minimum, and caps up to 254 keep messages in one byte
constexpr int kMaxDeltaG = 8000;
constexpr int kMaxCapG = 254;

#define DM_CK(call)                                  \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return DM_ERR_CUDA;   \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

double r_ab(double t, double a, double b)
{
    const double at = std::fabs(t);
    return at <= b ? a * at : at - b * (1.0 - a);
}

// r = r_{eps,delta} - r_{0, C + delta - eps delta}  (Eq. r-decompose)
double r_dc(double t, const dm_params& p)
{
    return r_ab(t, p.eps, p.delta) - r_ab(t, 0.0, p.C + p.delta - p.eps * p.delta);
}

bool is_int(double v, long long* out)
{
    const double rv = std::nearbyint(v);
    if (std::fabs(v - rv) > 1e-9) return false;
    *out = (long long)rv;
    return true;
}

// Taps of omega * r sampled at label distances (Sec. 2.2, Fig. 2).  Returns the
// number of distances below the cap (the window radius), or -1 if omega * r is
// not an integer table that reaches its cap within kRMax steps.
int build_taps(int omega, int L, const dm_params& p, int32_t* row)
{
    std::memset(row, 0, sizeof(int32_t) * dm::kTapW);
    long long cap;
    if (!is_int(omega * p.C, &cap)) return -1;
    int radius = 0;
    long long prev = 0;
    for (int t = 1; t < (L > dm::kRMax + 2 ? L : dm::kRMax + 2); ++t) {
        long long v;
        if (!is_int(omega * r_dc((double)t, p), &v)) return -1;
        if (v < prev || v > cap) return -1;
        if (v < cap) {
            if (t > dm::kRMax) return -1;
            radius = t;
        } else if (t <= dm::kRMax) {
            // at or beyond the cap: later taps are redundant, keep them at the cap
        }
        if (t <= dm::kRMax) row[t - 1] = (int32_t)(v < cap ? v : cap);
        prev = v;
    }
    row[dm::kTapP2] = (int32_t)cap;
    row[dm::kTapValid] = 1;
    return radius;
}

bool params_ok(const dm_params& p)
{
    if (p.struct_size != sizeof(dm_params)) return false;
    if (p.census_win != 3 && p.census_win != 5) return false;
    if (p.w_hi < 0 || p.w_hi > 255 || p.w_lo < 0 || p.w_lo > 255) return false;
    if (!(p.eps >= 0.0 && p.eps <= 1.0 && p.delta > 0.0 && p.C >= p.eps * p.delta)) return false;
    if (!(p.lambda_r >= 0.0 && p.alpha >= 0.0 && p.tau > 0.0 && p.sigma > 0.0 && p.h > 0.0))
        return false;
    if (p.warps < 1) return false;
    if (p.cost_bytes < 0 || p.cost_bytes > 2) return false;
    if (p.dmm_path < 0 || p.dmm_path > 3) return false;
    if (p.pd_launch < 0 || p.pd_launch > 2 || p.wait_test < 0) return false;
    return true;
}

dm::PdArgs pd_args(dm_ctx* c)
{
    dm::PdArgs a{};
    uint8_t* ws = c->ws;
    const dm::Layout& l = c->lay;
    a.H = c->H;
    a.W = c->W;
    a.L = c->L;
    a.cost = ws + l.cost;
    a.cost16 = c->cost_bytes == 2 ? reinterpret_cast<const uint16_t*>(ws + l.cost) : nullptr;
    a.wh = ws + l.wh;
    a.wv = ws + l.wv;
    a.alpha = (float)c->p.alpha;
    a.lambda_r = (float)c->p.lambda_r;
    a.tau = (float)c->p.tau;
    a.sigma = (float)c->p.sigma;
    a.h = (float)c->p.h;
    a.ap = (float)c->p.eps;
    a.bp = (float)c->p.delta;
    a.bq = (float)(c->p.C + c->p.delta - c->p.eps * c->p.delta);
    float* ua = reinterpret_cast<float*>(ws + l.u);
    float* ub = reinterpret_cast<float*>(ws + l.u_new);
    a.u = c->u_cur == 0 ? ua : ub;
    a.u_new = c->u_cur == 0 ? ub : ua;
    a.u0 = reinterpret_cast<float*>(ws + l.u0);
    a.s1 = reinterpret_cast<float*>(ws + l.s1);
    a.s2 = reinterpret_cast<float*>(ws + l.s2);
    a.lo = reinterpret_cast<float*>(ws + l.lo);
    a.hi = reinterpret_cast<float*>(ws + l.hi);
    float* pa[4] = {reinterpret_cast<float*>(ws + l.ph), reinterpret_cast<float*>(ws + l.pv),
                    reinterpret_cast<float*>(ws + l.qh), reinterpret_cast<float*>(ws + l.qv)};
    float* pb[4] = {reinterpret_cast<float*>(ws + l.ph2), reinterpret_cast<float*>(ws + l.pv2),
                    reinterpret_cast<float*>(ws + l.qh2), reinterpret_cast<float*>(ws + l.qv2)};
    float** in = c->pq_cur == 0 ? pa : pb;
    float** out = c->pq_cur == 0 ? pb : pa;
    a.ph = in[0];
    a.pv = in[1];
    a.qh = in[2];
    a.qv = in[3];
    a.ph2 = out[0];
    a.pv2 = out[1];
    a.qh2 = out[2];
    a.qv2 = out[3];
    a.costf = c->cost_f32;
    a.alpha_px = c->alpha_px;
    return a;
}

// one primal-dual state (u, p_h, p_v, q_h, q_v)
struct St {
    float* u;
    float* ph;
    float* pv;
    float* qh;
    float* qv;
};

St state_at(uint8_t* base, size_t slot)
{
    return {reinterpret_cast<float*>(base), reinterpret_cast<float*>(base + slot),
            reinterpret_cast<float*>(base + 2 * slot), reinterpret_cast<float*>(base + 3 * slot),
            reinterpret_cast<float*>(base + 4 * slot)};
}

St ws_set(dm_ctx* c, int which)
{
    uint8_t* ws = c->ws;
    const dm::Layout& l = c->lay;
    auto f = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
    if (which == 0) return {f(l.u), f(l.ph), f(l.pv), f(l.qh), f(l.qv)};
    return {f(l.u_new), f(l.ph2), f(l.pv2), f(l.qh2), f(l.qv2)};
}

dm::PdArgs pd_args_st(dm_ctx* c, const St& in, const St& out)
{
    dm::PdArgs a = pd_args(c);
    a.u = in.u;
    a.ph = in.ph;
    a.pv = in.pv;
    a.qh = in.qh;
    a.qv = in.qv;
    a.u_new = out.u;
    a.ph2 = out.ph;
    a.pv2 = out.pv;
    a.qh2 = out.qh;
    a.qv2 = out.qv;
    return a;
}

// Tape of the checkpointed forward: the state at every segment start (every
// ckpt_every iterations and every warp start, so no segment crosses a
// re-linearisation), slots to recompute one segment, two adjoint states, the
// per-pixel accumulators and the partial sums of d loss / d lambda_r.
struct TapePlan {
    std::vector<int> seg;         // first iteration of each segment
    std::vector<char> warp_first; // segment starts a warp
    std::vector<int> warp_seg;    // segment holding the start of its warp
    int iters = 0, max_len = 0;
    size_t slot = 0, off_ckpt = 0, off_seg = 0, off_adj = 0, off_acc = 0, off_part = 0, total = 0;
};

constexpr int kMaxTapeIters = 1 << 20;

int make_plan(const dm_ctx* c, int iters, int ckpt, TapePlan* tp)
{
    if (iters < 0 || iters > kMaxTapeIters || ckpt < 1) return DM_ERR_ARG;
    const int warps = c->p.warps, base = iters / warps, extra = iters % warps;
    std::vector<char> wstart(iters + 1, 0);
    for (int w = 0, k = 0; w < warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        if (nit > 0) wstart[k] = 1;
        k += nit;
    }
    tp->iters = iters;
    tp->seg.clear();
    tp->warp_first.clear();
    tp->warp_seg.clear();
    int cur_warp_seg = 0;
    for (int k = 0; k < iters; ++k) {
        if (k % ckpt == 0 || wstart[k]) {
            if (wstart[k]) cur_warp_seg = (int)tp->seg.size();
            tp->seg.push_back(k);
            tp->warp_first.push_back(wstart[k]);
            tp->warp_seg.push_back(cur_warp_seg);
        }
    }
    if (tp->seg.empty()) {  // no iterations: the tape holds the start state only
        tp->seg.push_back(0);
        tp->warp_first.push_back(0);
        tp->warp_seg.push_back(0);
    }
    tp->max_len = 0;
    for (size_t s = 0; s < tp->seg.size(); ++s) {
        const int end = s + 1 < tp->seg.size() ? tp->seg[s + 1] : iters;
        if (end - tp->seg[s] > tp->max_len) tp->max_len = end - tp->seg[s];
    }
    const size_t HW = (size_t)c->H * c->W;
    tp->slot = align_up(HW * sizeof(float), 256);
    const size_t st = 5 * tp->slot;
    tp->off_ckpt = 0;
    tp->off_seg = tp->off_ckpt + tp->seg.size() * st;
    tp->off_adj = tp->off_seg + (size_t)tp->max_len * st;
    tp->off_acc = tp->off_adj + 2 * st;
    tp->off_part = tp->off_acc + 4 * tp->slot;
    tp->total = tp->off_part + align_up(1024 * sizeof(double), 256);
    return DM_OK;
}

// an NVTX range over one C ABI stage (a no-op unless a profiler listens)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// the split Dual MM pass's counters
size_t pool_bytes(const dm_ctx*) { return dm::kPoolHead * sizeof(int32_t); }

int check_device_error(dm_ctx* c)
{
    int32_t err = 0;
    DM_CK(cudaMemcpyAsync(&err, c->ws + c->lay.err, sizeof(err), cudaMemcpyDeviceToHost,
                          c->stream));
    DM_CK(cudaStreamSynchronize(c->stream));
    if (err == 0) return DM_OK;
    // a dual outside the packed storage's range and a wait that gave up have
    // their own codes
    if ((err & dm::kDevErrRange) != 0) return DM_ERR_RANGE;
    if ((err & dm::kDevErrTimeout) != 0) {
        // cleared once reported: the barriers of the next one-launch
        // refinement give up as soon as they see it
        DM_CK(cudaMemsetAsync(c->ws + c->lay.err, 0, sizeof(int32_t), c->stream));
        DM_CK(cudaStreamSynchronize(c->stream));
        return DM_ERR_TIMEOUT;
    }
    return DM_ERR_DEVICE;
}

int ready(const dm_ctx* c)
{
    if (c == nullptr) return DM_ERR_ARG;
    if (c->ws == nullptr) return DM_ERR_STATE;
    return DM_OK;
}

// packed messages of the 16-bit kernel: 32 * np16 uint32 per chain node
size_t msg16_bytes(const dm_ctx* c)
{
    return align_up((size_t)c->H * c->W * 32 * c->np16 * sizeof(uint32_t), 256);
}

size_t base_bytes(const dm_ctx* c) { return align_up((size_t)c->H * c->W * 4, 256); }

dm::Dmm16Args dm16_args(dm_ctx* c, int which)
{
    dm::Dmm16Args a{};
    uint8_t* ws = c->ws;
    uint8_t* lh = ws + c->lay.lam_h;
    uint8_t* lv = ws + c->lay.lam_v;
    uint8_t* in = which == 0 ? lv : lh;
    uint8_t* out = which == 0 ? lh : lv;
    a.which = which;
    a.H = c->H;
    a.W = c->W;
    a.L = c->L;
    a.cost = ws + c->lay.cost;
    a.cost16 = c->cost_bytes == 2 ? reinterpret_cast<const uint16_t*>(ws + c->lay.cost) : nullptr;
    a.base_in = reinterpret_cast<const int32_t*>(in);
    a.delta_in = in + base_bytes(c);
    a.base_out = reinterpret_cast<int32_t*>(out);
    a.delta_out = out + base_bytes(c);
    a.wedge = ws + (which == 0 ? c->lay.wh : c->lay.wv);
    a.fmsg = reinterpret_cast<uint32_t*>(ws + c->lay.fmsg);
    a.bmsg = reinterpret_cast<uint32_t*>(ws + c->lay.bmsg);
    a.fofs = reinterpret_cast<int32_t*>(ws + c->lay.fmsg + msg16_bytes(c));
    a.bofs = reinterpret_cast<int32_t*>(ws + c->lay.bmsg + msg16_bytes(c));
    a.taps16 = reinterpret_cast<const uint32_t*>(ws + c->lay.taps16);
    a.err = reinterpret_cast<int32_t*>(ws + c->lay.err);
    const int n = which == 0 ? c->W : c->H;
    int cap = 1;
    while (cap < n) cap <<= 1;
    a.seg_cap = (cap + 1 + 7) & ~7;  // keeps the second array 16-byte aligned
    return a;
}

// arguments of a packed pass on the context's kernel: the lane-group kernel
// keeps 8-bit messages [chains][n][16 gsz] with the int32 offsets after them
dm::Dmm16Args pass16_args(dm_ctx* c, int which)
{
    dm::Dmm16Args a = dm16_args(c, which);
    if (c->use_g) {
        const size_t msg = align_up((size_t)c->H * c->W * 16 * c->gsz, 256);
        a.fofs = reinterpret_cast<int32_t*>(c->ws + c->lay.fmsg + msg);
        a.bofs = reinterpret_cast<int32_t*>(c->ws + c->lay.bmsg + msg);
    }
    return a;
}

int run_pass16(dm_ctx* c, int which, uint16_t* labels, long long* lb)
{
    dm::Dmm16Args a = pass16_args(c, which);
    a.labels = labels;
    a.lb = lb;
    if (c->use_g) {
        if (c->pool_g) a.pool = reinterpret_cast<int32_t*>(c->ws + c->lay.pool);
        DM_CK(dm::launch_dmg_pass(a, c->gsz, c->radius, c->delta_bytes, c->stream));
        c->launches += dm::dmg_pass_kernels(a, c->gsz);
        return DM_OK;
    }
    DM_CK(dm::launch_dmm16_pass(a, c->np16, c->radius, c->delta_bytes, c->stream));
    c->launches += 1;
    return DM_OK;
}

// kernel and storage of the duals for a new cost volume whose values are <=
// cost_max: the packed 16-bit kernel needs every dual delta, at most
// max(c) + 2 (omega C + 1), to stay below its 16-bit infinity; the int32 kernel
// needs (max(c) + 4 omega C) times the chain length below 2^30
void set_path(dm_ctx* c, int cost_max, bool user_weights)
{
    const int p2 = user_weights ? c->p2_all : c->p2_used;
    c->user_weights = user_weights;
    c->cost_max = cost_max;
    c->use16 = c->can16 && c->minorant == 0 && cost_max + 2 * (p2 + 1) <= kMaxDelta16;
    c->use_g = c->use16 && c->can_g && cost_max + 2 * (p2 + 1) <= kMaxDeltaG && p2 <= kMaxCapG;
    c->delta_bytes = (cost_max + 2 * (p2 + 1) <= 255) ? 1 : 2;
}

int choose_path(dm_ctx* c, int cost_max, bool user_weights)
{
    const long long n = (c->H > c->W ? c->H : c->W) + 1;
    if (c->discrete_ok && ((long long)cost_max + 4LL * c->p2_all) * n >= (1LL << 30))
        return DM_ERR_RANGE;
    set_path(c, cost_max, user_weights);
    if (!c->discrete_ok) return DM_OK;  // weights only feed the continuous stage
    DM_CK(dm::launch_validate_edges(c->ws + c->lay.wh, c->ws + c->lay.wv, c->H, c->W,
                                    reinterpret_cast<const int32_t*>(c->ws + c->lay.taps),
                                    reinterpret_cast<int32_t*>(c->ws + c->lay.err), c->stream));
    c->launches += 1;
    return DM_OK;
}

int run_pass(dm_ctx* c, int which, uint16_t* labels, long long* lb)
{
    if (c->use16) return run_pass16(c, which, labels, lb);
    dm::DmmArgs a{};
    uint8_t* ws = c->ws;
    a.which = which;
    a.H = c->H;
    a.W = c->W;
    a.L = c->L;
    a.KP = c->KP;
    a.cost = ws + c->lay.cost;
    a.cost16 = c->cost_bytes == 2 ? reinterpret_cast<const uint16_t*>(ws + c->lay.cost) : nullptr;
    int32_t* lh = reinterpret_cast<int32_t*>(ws + c->lay.lam_h);
    int32_t* lv = reinterpret_cast<int32_t*>(ws + c->lay.lam_v);
    a.lam_in = which == 0 ? lv : lh;
    a.lam_out = which == 0 ? lh : lv;
    a.wedge = ws + (which == 0 ? c->lay.wh : c->lay.wv);
    a.fmsg = reinterpret_cast<int32_t*>(ws + c->lay.fmsg);
    a.bmsg = reinterpret_cast<int32_t*>(ws + c->lay.bmsg);
    a.taps = reinterpret_cast<const int32_t*>(ws + c->lay.taps);
    a.err = reinterpret_cast<int32_t*>(ws + c->lay.err);
    a.labels = labels;
    a.lb = lb;
    a.minorant = c->minorant;
    a.max_pass = c->max_pass;
    a.gamma_num = c->gamma_num;
    a.gamma_den = c->gamma_den;
    DM_CK(dm::launch_dmm_pass(a, c->lpt, c->radius, c->stream));
    c->launches += 1;
    return DM_OK;
}

// census, edge weights and cost volume of a new pair (the duals are left alone)
int census_cost(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, bool mirror = false)
{
    uint8_t* ws = ctx->ws;
    uint32_t* census = reinterpret_cast<uint32_t*>(ws + ctx->lay.census);
    const int maxc = ctx->p.census_win * ctx->p.census_win - 1;
    DM_CK(dm::launch_census_edges(d_left, d_right, ctx->H, ctx->W, ctx->p.census_win,
                                  ctx->p.edge_threshold, ctx->p.w_hi, ctx->p.w_lo, census,
                                  ws + ctx->lay.wh, ws + ctx->lay.wv, mirror, ctx->stream));
    DM_CK(dm::launch_cost(census, ctx->H, ctx->W, ctx->L, maxc, ws + ctx->lay.cost,
                          ctx->cost_bytes, ctx->stream));
    ctx->launches += 2;
    ctx->have_cost = true;
    ctx->have_weights = true;
    ctx->cost_f32 = nullptr;
    ctx->tape_valid = false;
    return choose_path(ctx, maxc, false);
}

}  // namespace

namespace dm {
namespace ctxops {
PdArgs pd_args(dm_ctx* c) { return ::pd_args(c); }
Dmm16Args dm16_args(dm_ctx* c, int which) { return ::pass16_args(c, which); }
int run_pass(dm_ctx* c, int which, uint16_t* labels, long long* lb)
{
    return ::run_pass(c, which, labels, lb);
}
void predict_path(dm_ctx* c, int cost_max) { ::set_path(c, cost_max, false); }
size_t base_bytes(const dm_ctx* c) { return ::base_bytes(c); }
}  // namespace ctxops
}  // namespace dm

namespace dm {
// Penalty taps of one edge weight and the parameter check (shared with the
// allocation-free entry point).
int penalty_taps(int omega, int L, const dm_params& p, int32_t* row)
{
    return build_taps(omega, L, p, row);
}
bool params_valid(const dm_params& p) { return params_ok(p); }
}  // namespace dm

extern "C" {

DM_API int dm_default_params(dm_params* p)
{
    if (p == nullptr) return DM_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(dm_params);
    p->census_win = 5;
    p->edge_threshold = 16;
    p->w_hi = 8;
    p->w_lo = 4;
    p->eps = 0.25;
    p->delta = 1.0;
    p->C = 2.0;
    p->lambda_r = 1.0;
    p->alpha = 1.0;
    p->tau = 0.35;
    p->sigma = 0.35;
    p->h = 1.0;
    p->warps = 5;
    return DM_OK;
}

DM_API int dm_create(int H, int W, int L, const dm_params* p, dm_ctx** out)
{
    if (out == nullptr || p == nullptr) return DM_ERR_ARG;
    *out = nullptr;
    if (H < 1 || W < 1 || L < 2 || L > 256) return DM_ERR_ARG;
    if ((long long)H * W * L >= (1LL << 31) || H > 65535 || W > 65535) return DM_ERR_ARG;
    if (!params_ok(*p)) return DM_ERR_ARG;
    dm_ctx* c = new (std::nothrow) dm_ctx();
    if (c == nullptr) return DM_ERR_ARG;
    c->H = H;
    c->W = W;
    c->L = L;
    c->p = *p;
    c->cost_bytes = p->cost_bytes == 2 ? 2 : 1;
    c->lpt = L <= 32 ? 1 : (L <= 64 ? 2 : (L <= 128 ? 4 : 8));
    c->KP = 32 * c->lpt;
    c->taps.assign(256 * dm::kTapW, 0);
    int radius = 1;
    for (int om = 0; om < 256; ++om) {
        const int r = build_taps(om, L, *p, &c->taps[om * dm::kTapW]);
        if (r < 0 && (om == p->w_hi || om == p->w_lo)) c->discrete_ok = false;
        if (r > radius) radius = r;
    }
    c->radius = radius;
    c->np16 = L <= 64 ? 1 : (L <= 128 ? 2 : 4);
    c->taps16.assign(256 * dm::kTapW, 0u);
    for (int om = 0; om < 256; ++om) {
        const int32_t* row = &c->taps[om * dm::kTapW];
        if (!row[dm::kTapValid]) continue;
        // packed row: {T1, T2, P2, valid, T3, T4, 0, 0}, taps in both 16-bit halves
        uint32_t* r16 = &c->taps16[om * dm::kTapW];
        r16[0] = ((uint32_t)row[0] & 0xffffu) * 0x10001u;
        r16[1] = ((uint32_t)row[1] & 0xffffu) * 0x10001u;
        r16[2] = (uint32_t)row[dm::kTapP2];
        r16[3] = 1u;
        r16[4] = ((uint32_t)row[2] & 0xffffu) * 0x10001u;
        r16[5] = ((uint32_t)row[3] & 0xffffu) * 0x10001u;
        if (row[dm::kTapP2] > c->p2_all) c->p2_all = row[dm::kTapP2];
        if ((om == p->w_hi || om == p->w_lo) && row[dm::kTapP2] > c->p2_used)
            c->p2_used = row[dm::kTapP2];
    }
    // the 16-bit kernel stages each unary row as four async copies of L/4 bytes
    // (uint8 deltas) or L/2 bytes (int16), so L must be a multiple of 16
    c->can16 = c->discrete_ok && p->dmm_path != 1 && (L % 16) == 0 && c->p2_all <= 8000 &&
               H <= 8192 && W <= 8192;
    c->can_g = c->can16 && p->dmm_path != 2;
    c->pool_g = p->dmm_path == 0;
    c->gsz = L <= 16 ? 1 : (L <= 32 ? 2 : (L <= 64 ? 4 : (L <= 128 ? 8 : 16)));
    // workspace layout
    dm::Layout& l = c->lay;
    size_t tot = 0;
    auto add = [&](size_t bytes) {
        const size_t off = align_up(tot, 256);
        tot = off + bytes;
        return off;
    };
    const size_t HW = (size_t)H * W, HWL = HW * L;
    l.cost = add(HWL * c->cost_bytes);
    l.census = add(2 * HW * sizeof(uint32_t));
    l.img = add(2 * HW);
    l.wh = add(HW);
    l.wv = add(HW);
    l.lam_h = add(HWL * sizeof(int32_t));
    l.lam_v = add(HWL * sizeof(int32_t));
    // message scratch: int32 messages of the int32 kernel, or packed messages
    // plus one int32 offset per node for the 16-bit kernel
    const size_t msg32 = HW * c->KP * sizeof(int32_t);
    const size_t msg16 = align_up(HW * 32 * c->np16 * sizeof(uint32_t), 256) + HW * sizeof(int32_t);
    l.fmsg = add(msg32 > msg16 ? msg32 : msg16);
    l.bmsg = add(msg32 > msg16 ? msg32 : msg16);
    l.labels = add(HW * sizeof(uint16_t));
    l.lb = add(kMaxIters * sizeof(long long));
    l.taps = add(256 * dm::kTapW * sizeof(int32_t));
    l.taps16 = add(256 * dm::kTapW * sizeof(uint32_t));
    l.u = add(HW * 4);
    l.u_new = add(HW * 4);
    l.u0 = add(HW * 4);
    l.s1 = add(HW * 4);
    l.s2 = add(HW * 4);
    l.lo = add(HW * 4);
    l.hi = add(HW * 4);
    l.ph = add(HW * 4);
    l.pv = add(HW * 4);
    l.qh = add(HW * 4);
    l.qv = add(HW * 4);
    l.ph2 = add(HW * 4);
    l.pv2 = add(HW * 4);
    l.qh2 = add(HW * 4);
    l.qv2 = add(HW * 4);
    l.epart = add(1024 * sizeof(double));
    l.err = add(sizeof(int32_t));
    l.bar = add(sizeof(uint32_t));
    l.pool = add(pool_bytes(c));
    l.total = align_up(tot, 256);
    *out = c;
    return DM_OK;
}

DM_API int dm_destroy(dm_ctx* ctx)
{
    if (ctx != nullptr) {
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->graph) cudaGraphDestroy(ctx->graph);
    }
    delete ctx;
    return DM_OK;
}

DM_API int dm_workspace_bytes(const dm_ctx* ctx, size_t* bytes)
{
    if (ctx == nullptr || bytes == nullptr) return DM_ERR_ARG;
    *bytes = ctx->lay.total;
    return DM_OK;
}

DM_API int dm_bind_workspace(dm_ctx* ctx, void* d_workspace, size_t bytes)
{
    if (ctx == nullptr || d_workspace == nullptr) return DM_ERR_ARG;
    if (bytes < ctx->lay.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0)
        return DM_ERR_WORKSPACE;
    ctx->ws = static_cast<uint8_t*>(d_workspace);
    ctx->ws_bytes = bytes;
    ctx->have_cost = ctx->have_labels = ctx->have_u = ctx->have_weights = false;
    ctx->tape_valid = false;
    ctx->u_cur = 0;
    ctx->last_iters = 0;
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.taps, ctx->taps.data(),
                          ctx->taps.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.taps16, ctx->taps16.data(),
                          ctx->taps16.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                          ctx->stream));
    DM_CK(cudaMemsetAsync(ctx->ws + ctx->lay.err, 0, sizeof(int32_t), ctx->stream));
    DM_CK(cudaMemsetAsync(ctx->ws + ctx->lay.pool, 0, pool_bytes(ctx), ctx->stream));
    DM_CK(cudaStreamSynchronize(ctx->stream));
    return DM_OK;
}

DM_API int dm_set_stream(dm_ctx* ctx, void* stream)
{
    if (ctx == nullptr) return DM_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return DM_OK;
}

DM_API int dm_set_cost_volume_u16(dm_ctx* ctx, const uint16_t* d_cost, const uint8_t* d_wh,
                                  const uint8_t* d_wv, int cost_max)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_cost == nullptr || d_wh == nullptr || d_wv == nullptr) return DM_ERR_ARG;
    if (cost_max < 0 || cost_max > 65535 || (reinterpret_cast<uintptr_t>(d_cost) & 1)) return DM_ERR_ARG;
    if (ctx->cost_bytes != 2) return DM_ERR_STATE;
    const size_t HW = (size_t)ctx->H * ctx->W;
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.cost, d_cost, HW * ctx->L * sizeof(uint16_t),
                          cudaMemcpyDeviceToDevice, ctx->stream));
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.wh, d_wh, HW, cudaMemcpyDeviceToDevice, ctx->stream));
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.wv, d_wv, HW, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->have_cost = true;
    ctx->have_weights = true;
    ctx->cost_f32 = nullptr;
    ctx->tape_valid = false;
    if ((rc = choose_path(ctx, cost_max, true))) return rc;
    return dm_reset_duals(ctx);
}

DM_API int dm_reset_duals(dm_ctx* ctx)
{
    int rc = ready(ctx);
    if (rc) return rc;
    const size_t HWL = (size_t)ctx->H * ctx->W * ctx->L;
    if (!(ctx->use16 && ctx->have_cost)) {
        DM_CK(cudaMemsetAsync(ctx->ws + ctx->lay.lam_v, 0, HWL * sizeof(int32_t), ctx->stream));
        DM_CK(cudaMemsetAsync(ctx->ws + ctx->lay.lam_h, 0, HWL * sizeof(int32_t), ctx->stream));
    } else {
        // lambda_h = 0 in the packed storage (a base and deltas); the 16-bit path
        // keeps c + lambda_v in place of lambda_v: c for a cold start
        DM_CK(cudaMemsetAsync(ctx->ws + ctx->lay.lam_h, 0,
                              base_bytes(ctx) + HWL * ctx->delta_bytes, ctx->stream));
        uint8_t* reg = ctx->ws + ctx->lay.lam_v;
        DM_CK(dm::launch_theta_h_init(ctx->ws + ctx->lay.cost, ctx->cost_bytes,
                                      reinterpret_cast<int32_t*>(reg),
                                      reg + base_bytes(ctx), ctx->delta_bytes,
                                      (long long)ctx->H * ctx->W, ctx->L, ctx->stream));
        // uint8 costs into uint8 deltas are a copy, not a kernel
        if (!(ctx->cost_bytes == 1 && ctx->delta_bytes == 1)) ctx->launches += 1;
    }
    ctx->have_labels = false;
    return DM_OK;
}

DM_API int dm_cost_volume(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right)
{
    const Range range("dm_cost_volume");
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_left == nullptr || d_right == nullptr) return DM_ERR_ARG;
    if ((rc = census_cost(ctx, d_left, d_right))) return rc;
    return dm_reset_duals(ctx);
}

DM_API int dm_cost_volume_warm(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right)
{
    const Range range("dm_cost_volume_warm");
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_left == nullptr || d_right == nullptr) return DM_ERR_ARG;
    const bool warm = ctx->have_cost && ctx->cost_f32 == nullptr && ctx->discrete_ok;
    if (!warm) return dm_cost_volume(ctx, d_left, d_right);
    const long long n_px = (long long)ctx->H * ctx->W;
    uint8_t* reg = ctx->ws + ctx->lay.lam_v;
    int32_t* lam_v32 = reinterpret_cast<int32_t*>(ctx->ws + ctx->lay.lam_h);
    const bool was16 = ctx->use16;
    if (was16) {
        // lambda_v = (c + lambda_v) - c with the previous frame's c, as int32 in the
        // lambda_h region (the next horizontal pass overwrites it)
        DM_CK(dm::launch_duals_to_i32(reinterpret_cast<const int32_t*>(reg), reg + base_bytes(ctx),
                                      ctx->delta_bytes, ctx->ws + ctx->lay.cost, ctx->cost_bytes,
                                      n_px, ctx->L, lam_v32, ctx->stream));
        ctx->launches += 1;
    }
    if ((rc = census_cost(ctx, d_left, d_right))) return rc;
    if (ctx->use16) {
        const int32_t* src = was16 ? lam_v32 : reinterpret_cast<const int32_t*>(reg);
        if (!was16) {
            // int32 lambda_v -> the lambda_h region, then c + lambda_v into place
            DM_CK(cudaMemcpyAsync(lam_v32, reg, (size_t)n_px * ctx->L * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, ctx->stream));
            src = lam_v32;
        }
        DM_CK(dm::launch_theta_h_from_i32(src, ctx->ws + ctx->lay.cost, ctx->cost_bytes,
                                          reinterpret_cast<int32_t*>(reg), reg + base_bytes(ctx),
                                          ctx->delta_bytes, n_px, ctx->L,
                                          reinterpret_cast<int32_t*>(ctx->ws + ctx->lay.err),
                                          ctx->stream));
        ctx->launches += 1;
    } else if (was16) {
        DM_CK(cudaMemcpyAsync(reg, lam_v32, (size_t)n_px * ctx->L * sizeof(int32_t),
                              cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ctx->have_labels = false;
    return DM_OK;
}

DM_API int dm_set_cost_volume(dm_ctx* ctx, const uint8_t* d_cost, const uint8_t* d_wh,
                              const uint8_t* d_wv)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_cost == nullptr || d_wh == nullptr || d_wv == nullptr) return DM_ERR_ARG;
    if (ctx->cost_bytes != 1) return DM_ERR_STATE;
    const size_t HW = (size_t)ctx->H * ctx->W;
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.cost, d_cost, HW * ctx->L, cudaMemcpyDeviceToDevice,
                          ctx->stream));
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.wh, d_wh, HW, cudaMemcpyDeviceToDevice, ctx->stream));
    DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.wv, d_wv, HW, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->have_cost = true;
    ctx->have_weights = true;
    ctx->cost_f32 = nullptr;
    ctx->tape_valid = false;
    if ((rc = choose_path(ctx, 255, true))) return rc;
    return dm_reset_duals(ctx);
}

DM_API int dm_discrete_pass(dm_ctx* ctx, int which)
{
    if (ctx == nullptr || (which != 0 && which != 1) || !ctx->discrete_ok) return DM_ERR_ARG;
    int rc = ready(ctx);
    if (rc) return rc;
    if (!ctx->have_cost || ctx->cost_f32 != nullptr) return DM_ERR_STATE;
    return run_pass(ctx, which, nullptr, nullptr);
}

DM_API int dm_discrete(dm_ctx* ctx, int iters, int64_t* h_lb)
{
    const Range range("dm_discrete");
    if (ctx == nullptr || iters < 1 || iters > kMaxIters || !ctx->discrete_ok) return DM_ERR_ARG;
    int rc = ready(ctx);
    if (rc) return rc;
    if (!ctx->have_cost || ctx->cost_f32 != nullptr) return DM_ERR_STATE;
    long long* lb = reinterpret_cast<long long*>(ctx->ws + ctx->lay.lb);
    uint16_t* labels = reinterpret_cast<uint16_t*>(ctx->ws + ctx->lay.labels);
    DM_CK(cudaMemsetAsync(lb, 0, iters * sizeof(long long), ctx->stream));
    for (int t = 0; t < iters; ++t) {
        if ((rc = run_pass(ctx, 0, nullptr, nullptr))) return rc;
        if ((rc = run_pass(ctx, 1, t == iters - 1 ? labels : nullptr, lb + t))) return rc;
    }
    ctx->have_labels = true;
    ctx->last_iters = iters;
    if (h_lb != nullptr) {
        DM_CK(cudaMemcpyAsync(h_lb, lb, iters * sizeof(long long), cudaMemcpyDeviceToHost,
                              ctx->stream));
        return check_device_error(ctx);
    }
    return DM_OK;
}

DM_API int dm_refine(dm_ctx* ctx, int iters, const float* d_u0)
{
    const Range range("dm_refine");
    int rc = ready(ctx);
    if (rc) return rc;
    if (iters < 0) return DM_ERR_ARG;
    if (!ctx->have_cost) return DM_ERR_STATE;
    if (d_u0 == nullptr && !ctx->have_labels) return DM_ERR_STATE;
    const int n = ctx->H * ctx->W;
    ctx->u_cur = 0;
    ctx->pq_cur = 0;
    dm::PdArgs a = pd_args(ctx);
    if (d_u0 != nullptr)
        DM_CK(cudaMemcpyAsync(a.u, d_u0, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    const int warps = ctx->p.warps;
    dm::PdResPlan plan{};
    if (ctx->p.pd_launch == 0 && dm::pd_res_plan(ctx->H, ctx->W, &plan)) {
        // every iteration in one cooperative launch, the state in shared memory
        // (pd_res_kernel)
        dm::PdResArgs r{};
        r.a = a;
        r.labels = d_u0 != nullptr ? nullptr
                                   : reinterpret_cast<const uint16_t*>(ctx->ws + ctx->lay.labels);
        r.iters = iters;
        r.warps = warps;
        r.nx = plan.nx;
        r.ny = plan.ny;
        r.RW = plan.RW;
        r.RH = plan.RH;
        r.K = plan.K;
        r.EW = plan.EW;
        r.EH = plan.EH;
        r.TR = plan.TR;
        r.bar = reinterpret_cast<unsigned*>(ctx->ws + ctx->lay.bar);
        r.err = reinterpret_cast<int32_t*>(ctx->ws + ctx->lay.err);
        r.wait_skew = ctx->p.wait_test;
        r.wait_ns = ctx->p.wait_test > 0 ? 20000000LL : 1000000000LL;
        DM_CK(cudaMemsetAsync(r.bar, 0, sizeof(unsigned), ctx->stream));
        DM_CK(dm::launch_pd_res(r, plan, ctx->stream));
        ctx->launches += 1;
        ctx->u_cur = ctx->pq_cur = dm::pd_res_result_set(iters, warps, plan.K);
        ctx->have_u = true;
        return DM_OK;
    }
    if (ctx->p.pd_launch == 2) {
        // every iteration in one cooperative launch (pd_run_kernel)
        dm::PdRunArgs r{};
        r.set[0] = a;
        ctx->u_cur = ctx->pq_cur = 1;
        r.set[1] = pd_args(ctx);
        r.labels = d_u0 != nullptr ? nullptr
                                   : reinterpret_cast<const uint16_t*>(ctx->ws + ctx->lay.labels);
        r.iters = iters;
        r.warps = warps;
        r.bar = reinterpret_cast<unsigned*>(ctx->ws + ctx->lay.bar);
        r.err = reinterpret_cast<int32_t*>(ctx->ws + ctx->lay.err);
        r.bar_skew = ctx->p.wait_test;
        r.wait_ns = ctx->p.wait_test > 0 ? 20000000LL : 1000000000LL;
        DM_CK(cudaMemsetAsync(r.bar, 0, sizeof(unsigned), ctx->stream));
        DM_CK(dm::launch_pd_run(r, ctx->stream));
        ctx->launches += 1;
        ctx->u_cur = ctx->pq_cur = iters & 1;
        ctx->have_u = true;
        return DM_OK;
    }
    if (d_u0 == nullptr)
        DM_CK(dm::launch_init_u_from_labels(
            reinterpret_cast<const uint16_t*>(ctx->ws + ctx->lay.labels), a.u, n, ctx->stream));
    for (float* s : {a.ph, a.pv, a.qh, a.qv, a.ph2, a.pv2, a.qh2, a.qv2})
        DM_CK(dm::launch_zero_f32(s, n, ctx->stream));
    ctx->launches += (d_u0 != nullptr ? 0 : 1) + 8;
    const int base = iters / warps, extra = iters % warps;
    for (int w = 0; w < warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        a = pd_args(ctx);
        DM_CK(dm::launch_linearise(a, ctx->stream));
        ctx->launches += 1;
        for (int it = 0; it < nit; ++it) {
            a = pd_args(ctx);
            DM_CK(dm::launch_pd_iter(a, ctx->stream));
            ctx->launches += 1;
            ctx->u_cur ^= 1;
            ctx->pq_cur ^= 1;
        }
    }
    ctx->have_u = true;
    return DM_OK;
}

DM_API int dm_set_cost_volume_f32(dm_ctx* ctx, const float* d_cost, const uint8_t* d_wh,
                                  const uint8_t* d_wv)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_cost == nullptr || (d_wh == nullptr) != (d_wv == nullptr)) return DM_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_cost) & 3) return DM_ERR_ARG;
    if (d_wh != nullptr) {
        const size_t HW = (size_t)ctx->H * ctx->W;
        DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.wh, d_wh, HW, cudaMemcpyDeviceToDevice,
                              ctx->stream));
        DM_CK(cudaMemcpyAsync(ctx->ws + ctx->lay.wv, d_wv, HW, cudaMemcpyDeviceToDevice,
                              ctx->stream));
        ctx->have_weights = true;
    }
    if (!ctx->have_weights) return DM_ERR_STATE;
    ctx->cost_f32 = d_cost;
    ctx->have_cost = true;
    ctx->tape_valid = false;
    return DM_OK;
}

DM_API int dm_set_data_weights(dm_ctx* ctx, const float* d_alpha)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(d_alpha) & 3) return DM_ERR_ARG;
    ctx->alpha_px = d_alpha;
    ctx->tape_valid = false;
    return DM_OK;
}

DM_API int dm_set_lambda_r(dm_ctx* ctx, double lambda_r)
{
    if (ctx == nullptr || !(lambda_r >= 0.0) || !std::isfinite(lambda_r)) return DM_ERR_ARG;
    ctx->p.lambda_r = lambda_r;
    ctx->tape_valid = false;
    return DM_OK;
}

DM_API int dm_tape_bytes(const dm_ctx* ctx, int iters, int ckpt_every, size_t* bytes)
{
    if (ctx == nullptr || bytes == nullptr) return DM_ERR_ARG;
    TapePlan tp;
    int rc = make_plan(ctx, iters, ckpt_every, &tp);
    if (rc) return rc;
    *bytes = tp.total;
    return DM_OK;
}

DM_API int dm_refine_tape(dm_ctx* ctx, int iters, int ckpt_every, const float* d_u0, void* d_tape,
                          size_t tape_bytes)
{
    const Range range("dm_refine_tape");
    int rc = ready(ctx);
    if (rc) return rc;
    TapePlan tp;
    if ((rc = make_plan(ctx, iters, ckpt_every, &tp))) return rc;
    if (!ctx->have_cost) return DM_ERR_STATE;
    if (d_u0 == nullptr && !ctx->have_labels) return DM_ERR_STATE;
    if (d_tape == nullptr || tape_bytes < tp.total ||
        (reinterpret_cast<uintptr_t>(d_tape) & 255) != 0)
        return DM_ERR_WORKSPACE;
    ctx->tape_valid = false;
    const int n = ctx->H * ctx->W;
    uint8_t* T = static_cast<uint8_t*>(d_tape);
    auto ckpt = [&](size_t s) { return state_at(T + tp.off_ckpt + s * 5 * tp.slot, tp.slot); };
    St cur = ckpt(0);
    if (d_u0 != nullptr)
        DM_CK(cudaMemcpyAsync(cur.u, d_u0, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    else {
        DM_CK(dm::launch_init_u_from_labels(
            reinterpret_cast<const uint16_t*>(ctx->ws + ctx->lay.labels), cur.u, n, ctx->stream));
        ctx->launches += 1;
    }
    DM_CK(cudaMemsetAsync(cur.ph, 0, 4 * tp.slot, ctx->stream));
    int curset = 2;  // 0, 1: workspace sets, 2: a checkpoint slot
    size_t s_next = 1;
    const int warps = ctx->p.warps, base = iters / warps, extra = iters % warps;
    for (int w = 0, k = 0; w < warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        if (nit == 0) continue;
        DM_CK(dm::launch_linearise(pd_args_st(ctx, cur, cur), ctx->stream));
        ctx->launches += 1;
        for (int it = 0; it < nit; ++it, ++k) {
            St out;
            int outset;
            if (s_next < tp.seg.size() && tp.seg[s_next] == k + 1) {
                out = ckpt(s_next++);
                outset = 2;
            } else {
                outset = curset == 0 ? 1 : 0;
                out = ws_set(ctx, outset);
            }
            DM_CK(dm::launch_pd_iter(pd_args_st(ctx, cur, out), ctx->stream));
            ctx->launches += 1;
            cur = out;
            curset = outset;
        }
    }
    if (curset == 2) {  // no iterations: the start state becomes the current one
        const St a = ws_set(ctx, 0);
        float* src[5] = {cur.u, cur.ph, cur.pv, cur.qh, cur.qv};
        float* dst[5] = {a.u, a.ph, a.pv, a.qh, a.qv};
        for (int j = 0; j < 5; ++j)
            DM_CK(cudaMemcpyAsync(dst[j], src[j], n * sizeof(float), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
        curset = 0;
    }
    ctx->u_cur = ctx->pq_cur = curset;
    ctx->have_u = true;
    ctx->tape = d_tape;
    ctx->tape_bytes = tape_bytes;
    ctx->tape_iters = iters;
    ctx->tape_ckpt = ckpt_every;
    ctx->tape_valid = true;
    return DM_OK;
}

DM_API int dm_refine_backward(dm_ctx* ctx, const float* d_gu, void* d_tape, size_t tape_bytes,
                              float* d_gcost, float* d_galpha, double* d_glambda, float* d_gu0)
{
    const Range range("dm_refine_backward");
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_gu == nullptr) return DM_ERR_ARG;
    if (!ctx->tape_valid || d_tape != ctx->tape || tape_bytes != ctx->tape_bytes)
        return DM_ERR_STATE;
    TapePlan tp;
    if ((rc = make_plan(ctx, ctx->tape_iters, ctx->tape_ckpt, &tp))) return rc;
    const int n = ctx->H * ctx->W;
    const size_t HWL = (size_t)n * ctx->L;
    uint8_t* T = static_cast<uint8_t*>(d_tape);
    auto ckpt = [&](size_t s) { return state_at(T + tp.off_ckpt + s * 5 * tp.slot, tp.slot); };
    auto segst = [&](int j) { return state_at(T + tp.off_seg + (size_t)j * 5 * tp.slot, tp.slot); };
    St adj[2] = {state_at(T + tp.off_adj, tp.slot), state_at(T + tp.off_adj + 5 * tp.slot, tp.slot)};
    float* acc = reinterpret_cast<float*>(T + tp.off_acc);
    float* gu0 = acc;
    float* gs1 = reinterpret_cast<float*>(T + tp.off_acc + tp.slot);
    float* gs2 = reinterpret_cast<float*>(T + tp.off_acc + 2 * tp.slot);
    float* glam = reinterpret_cast<float*>(T + tp.off_acc + 3 * tp.slot);
    if (d_gcost != nullptr) DM_CK(cudaMemsetAsync(d_gcost, 0, HWL * sizeof(float), ctx->stream));
    if (d_galpha != nullptr) DM_CK(cudaMemsetAsync(d_galpha, 0, n * sizeof(float), ctx->stream));
    DM_CK(cudaMemsetAsync(acc, 0, 4 * tp.slot, ctx->stream));
    DM_CK(cudaMemcpyAsync(adj[0].u, d_gu, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    DM_CK(cudaMemsetAsync(adj[0].ph, 0, 4 * tp.slot, ctx->stream));
    int cur = 0;
    const dm::PdArgs P = pd_args(ctx);
    for (int s = (int)tp.seg.size() - 1; s >= 0; --s) {
        const int k0 = tp.seg[s];
        const int k1 = s + 1 < (int)tp.seg.size() ? tp.seg[s + 1] : tp.iters;
        const int len = k1 - k0;
        if (len <= 0) continue;
        const St wst = ckpt(tp.warp_seg[s]);
        DM_CK(dm::launch_linearise(pd_args_st(ctx, wst, wst), ctx->stream));
        ctx->launches += 1;
        auto st = [&](int j) { return j == 0 ? ckpt(s) : segst(j - 1); };
        for (int j = 0; j < len; ++j) {
            DM_CK(dm::launch_pd_iter(pd_args_st(ctx, st(j), st(j + 1)), ctx->stream));
            ctx->launches += 1;
        }
        for (int j = len - 1; j >= 0; --j) {
            const St in = st(j);
            dm::AdjArgs a{};
            a.H = ctx->H;
            a.W = ctx->W;
            a.L = ctx->L;
            a.wh = P.wh;
            a.wv = P.wv;
            a.lambda_r = P.lambda_r;
            a.tau = P.tau;
            a.sigma = P.sigma;
            a.h = P.h;
            a.ap = P.ap;
            a.bp = P.bp;
            a.bq = P.bq;
            a.u = in.u;
            a.un = st(j + 1).u;
            a.ph = in.ph;
            a.pv = in.pv;
            a.qh = in.qh;
            a.qv = in.qv;
            a.u0 = P.u0;
            a.s1 = P.s1;
            a.s2 = P.s2;
            a.lo = P.lo;
            a.hi = P.hi;
            a.ub = adj[cur].u;
            a.phb = adj[cur].ph;
            a.pvb = adj[cur].pv;
            a.qhb = adj[cur].qh;
            a.qvb = adj[cur].qv;
            a.ub2 = adj[cur ^ 1].u;
            a.phb2 = adj[cur ^ 1].ph;
            a.pvb2 = adj[cur ^ 1].pv;
            a.qhb2 = adj[cur ^ 1].qh;
            a.qvb2 = adj[cur ^ 1].qv;
            a.gu0 = gu0;
            a.gs1 = gs1;
            a.gs2 = gs2;
            a.glam = glam;
            DM_CK(dm::launch_pd_adjoint(a, ctx->stream));
            ctx->launches += 1;
            cur ^= 1;
        }
        if (tp.warp_first[s]) {
            dm::LinAdjArgs b{};
            b.H = ctx->H;
            b.W = ctx->W;
            b.L = ctx->L;
            b.cost = P.cost;
            b.cost16 = P.cost16;
            b.costf = P.costf;
            b.alpha_px = P.alpha_px;
            b.alpha = P.alpha;
            b.h = P.h;
            b.u0 = ckpt(s).u;
            b.gu0 = gu0;
            b.gs1 = gs1;
            b.gs2 = gs2;
            b.ub = adj[cur].u;
            b.gcost = d_gcost;
            b.galpha = d_galpha;
            DM_CK(dm::launch_lin_adjoint(b, ctx->stream));
            ctx->launches += 1;
        }
    }
    if (d_glambda != nullptr) {
        DM_CK(dm::launch_sum_f32(glam, n, reinterpret_cast<double*>(T + tp.off_part), d_glambda,
                                 ctx->stream));
        ctx->launches += 2;
    }
    if (d_gu0 != nullptr)
        DM_CK(cudaMemcpyAsync(d_gu0, adj[cur].u, n * sizeof(float), cudaMemcpyDeviceToDevice,
                              ctx->stream));
    return DM_OK;
}

DM_API int dm_jvp_bytes(const dm_ctx* ctx, size_t* bytes)
{
    if (ctx == nullptr || bytes == nullptr) return DM_ERR_ARG;
    *bytes = 15 * align_up((size_t)ctx->H * ctx->W * sizeof(float), 256);
    return DM_OK;
}

DM_API int dm_refine_jvp(dm_ctx* ctx, int iters, const float* d_u0, const float* d_du0,
                         const float* d_dcost, const float* d_dalpha, double dlambda, float* d_du,
                         void* d_scratch, size_t scratch_bytes)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (iters < 0 || d_du == nullptr || !std::isfinite(dlambda)) return DM_ERR_ARG;
    if (!ctx->have_cost) return DM_ERR_STATE;
    if (d_u0 == nullptr && !ctx->have_labels) return DM_ERR_STATE;
    size_t need;
    dm_jvp_bytes(ctx, &need);
    if (d_scratch == nullptr || scratch_bytes < need ||
        (reinterpret_cast<uintptr_t>(d_scratch) & 255) != 0)
        return DM_ERR_WORKSPACE;
    const int n = ctx->H * ctx->W;
    const size_t slot = align_up((size_t)n * sizeof(float), 256);
    uint8_t* S = static_cast<uint8_t*>(d_scratch);
    St tg[2] = {state_at(S, slot), state_at(S + 5 * slot, slot)};
    St lin = state_at(S + 10 * slot, slot);  // du0, ds1, ds2, dlo, dhi
    St cur = ws_set(ctx, 0);
    if (d_u0 != nullptr)
        DM_CK(cudaMemcpyAsync(cur.u, d_u0, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    else {
        DM_CK(dm::launch_init_u_from_labels(
            reinterpret_cast<const uint16_t*>(ctx->ws + ctx->lay.labels), cur.u, n, ctx->stream));
        ctx->launches += 1;
    }
    for (float* z : {cur.ph, cur.pv, cur.qh, cur.qv}) {
        DM_CK(dm::launch_zero_f32(z, n, ctx->stream));
        ctx->launches += 1;
    }
    if (d_du0 != nullptr)
        DM_CK(cudaMemcpyAsync(tg[0].u, d_du0, n * sizeof(float), cudaMemcpyDeviceToDevice,
                              ctx->stream));
    else
        DM_CK(cudaMemsetAsync(tg[0].u, 0, n * sizeof(float), ctx->stream));
    DM_CK(cudaMemsetAsync(tg[0].ph, 0, 4 * slot, ctx->stream));
    int cs = 0, ct = 0;
    auto jargs = [&](const St& fin, const St& fout, const St& tin, const St& tout) {
        dm::JvpArgs j{};
        j.f = pd_args_st(ctx, fin, fout);
        j.du = tin.u;
        j.dph = tin.ph;
        j.dpv = tin.pv;
        j.dqh = tin.qh;
        j.dqv = tin.qv;
        j.du2 = tout.u;
        j.dph2 = tout.ph;
        j.dpv2 = tout.pv;
        j.dqh2 = tout.qh;
        j.dqv2 = tout.qv;
        j.du0 = lin.u;
        j.ds1 = lin.ph;
        j.ds2 = lin.pv;
        j.dlo = lin.qh;
        j.dhi = lin.qv;
        j.dcost = d_dcost;
        j.dalpha = d_dalpha;
        j.dlambda = (float)dlambda;
        return j;
    };
    const int warps = ctx->p.warps, base = iters / warps, extra = iters % warps;
    for (int w = 0; w < warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        if (nit == 0) continue;
        DM_CK(dm::launch_lin_jvp(jargs(ws_set(ctx, cs), ws_set(ctx, cs), tg[ct], tg[ct]),
                                 ctx->stream));
        ctx->launches += 1;
        for (int it = 0; it < nit; ++it) {
            DM_CK(dm::launch_pd_jvp(jargs(ws_set(ctx, cs), ws_set(ctx, cs ^ 1), tg[ct], tg[ct ^ 1]),
                                    ctx->stream));
            ctx->launches += 1;
            cs ^= 1;
            ct ^= 1;
        }
    }
    DM_CK(cudaMemcpyAsync(d_du, tg[ct].u, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->u_cur = ctx->pq_cur = cs;
    ctx->have_u = true;
    return DM_OK;
}

DM_API int dm_get_labels(dm_ctx* ctx, uint16_t* d_labels)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_labels == nullptr) return DM_ERR_ARG;
    if (!ctx->have_labels) return DM_ERR_STATE;
    DM_CK(cudaMemcpyAsync(d_labels, ctx->ws + ctx->lay.labels,
                          (size_t)ctx->H * ctx->W * sizeof(uint16_t), cudaMemcpyDeviceToDevice,
                          ctx->stream));
    return DM_OK;
}

DM_API int dm_get_disparity(dm_ctx* ctx, float* d_u)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_u == nullptr) return DM_ERR_ARG;
    if (!ctx->have_u) return DM_ERR_STATE;
    dm::PdArgs a = pd_args(ctx);
    DM_CK(cudaMemcpyAsync(d_u, a.u, (size_t)ctx->H * ctx->W * sizeof(float),
                          cudaMemcpyDeviceToDevice, ctx->stream));
    return DM_OK;
}

DM_API int dm_get_duals(dm_ctx* ctx, int32_t* d_lam_h, int32_t* d_lam_v)
{
    int rc = ready(ctx);
    if (rc) return rc;
    const size_t bytes = (size_t)ctx->H * ctx->W * ctx->L * sizeof(int32_t);
    if (ctx->use16) {
        const long long npx = (long long)ctx->H * ctx->W;
        const size_t lay[2] = {ctx->lay.lam_h, ctx->lay.lam_v};
        int32_t* dst[2] = {d_lam_h, d_lam_v};
        for (int t = 0; t < 2; ++t) {
            if (dst[t] == nullptr) continue;
            const uint8_t* reg = ctx->ws + lay[t];
            DM_CK(dm::launch_duals_to_i32(reinterpret_cast<const int32_t*>(reg),
                                          reg + base_bytes(ctx), ctx->delta_bytes,
                                          t == 1 ? ctx->ws + ctx->lay.cost : nullptr,
                                          ctx->cost_bytes, npx, ctx->L, dst[t], ctx->stream));
            ctx->launches += 1;
        }
        return DM_OK;
    }
    if (d_lam_h)
        DM_CK(cudaMemcpyAsync(d_lam_h, ctx->ws + ctx->lay.lam_h, bytes, cudaMemcpyDeviceToDevice,
                              ctx->stream));
    if (d_lam_v)
        DM_CK(cudaMemcpyAsync(d_lam_v, ctx->ws + ctx->lay.lam_v, bytes, cudaMemcpyDeviceToDevice,
                              ctx->stream));
    return DM_OK;
}

DM_API int dm_get_cost_volume(dm_ctx* ctx, uint8_t* d_cost, uint8_t* d_wh, uint8_t* d_wv)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (!ctx->have_cost || (d_cost != nullptr && ctx->cost_f32 != nullptr)) return DM_ERR_STATE;
    const size_t HW = (size_t)ctx->H * ctx->W;
    if (d_cost)
        DM_CK(cudaMemcpyAsync(d_cost, ctx->ws + ctx->lay.cost, HW * ctx->L * ctx->cost_bytes,
                              cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_wh)
        DM_CK(cudaMemcpyAsync(d_wh, ctx->ws + ctx->lay.wh, HW, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_wv)
        DM_CK(cudaMemcpyAsync(d_wv, ctx->ws + ctx->lay.wv, HW, cudaMemcpyDeviceToDevice, ctx->stream));
    return DM_OK;
}

DM_API int dm_get_lower_bounds(dm_ctx* ctx, int64_t* h_lb, int n)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (h_lb == nullptr || n < 0 || n > ctx->last_iters) return DM_ERR_ARG;
    if (n > 0)
        DM_CK(cudaMemcpyAsync(h_lb, ctx->ws + ctx->lay.lb, n * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, ctx->stream));
    return check_device_error(ctx);
}

DM_API int dm_energy(dm_ctx* ctx, double* h_energy)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (h_energy == nullptr) return DM_ERR_ARG;
    if (!ctx->have_u) return DM_ERR_STATE;
    dm::PdArgs a = pd_args(ctx);
    const int nb = dm::energy_blocks(ctx->H, ctx->W);
    double* part = reinterpret_cast<double*>(ctx->ws + ctx->lay.epart);
    DM_CK(dm::launch_energy(a, ctx->p.eps, ctx->p.delta, ctx->p.C, part, nb, ctx->stream));
    ctx->launches += 1;
    std::vector<double> host(nb);
    DM_CK(cudaMemcpyAsync(host.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->stream));
    DM_CK(cudaStreamSynchronize(ctx->stream));
    double e = 0.0;
    for (int b = 0; b < nb; ++b) e += host[b];
    *h_energy = e;
    return check_device_error(ctx);
}

DM_API int dm_solve(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int dmm_iters,
                    int pd_iters, float* d_u)
{
    int rc;
    if ((rc = dm_cost_volume(ctx, d_left, d_right))) return rc;
    if ((rc = dm_discrete(ctx, dmm_iters, nullptr))) return rc;
    if ((rc = dm_refine(ctx, pd_iters, nullptr))) return rc;
    if (d_u != nullptr && (rc = dm_get_disparity(ctx, d_u))) return rc;
    return DM_OK;
}

DM_API int dm_capture(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int dmm_iters,
                      int pd_iters, float* d_u)
{
    const Range range("dm_capture");
    int rc = ready(ctx);
    if (rc) return rc;
    if (ctx->stream == nullptr) return DM_ERR_STATE;   // the legacy stream cannot be captured
    if (d_left == nullptr || d_right == nullptr || d_u == nullptr || dmm_iters < 1 ||
        pd_iters < 0)
        return DM_ERR_ARG;
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    DM_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    rc = dm_solve(ctx, d_left, d_right, dmm_iters, pd_iters, d_u);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rc != DM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != DM_OK ? rc : DM_ERR_CUDA;
    }
    ctx->graph = g;
    DM_CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
    return DM_OK;
}

DM_API int dm_replay(dm_ctx* ctx)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (ctx->graph_exec == nullptr) return DM_ERR_STATE;
    DM_CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    return DM_OK;
}

DM_API int dm_solve_next(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right,
                         int dmm_iters, int pd_iters, float* d_u)
{
    int rc;
    if ((rc = dm_cost_volume_warm(ctx, d_left, d_right))) return rc;
    if ((rc = dm_discrete(ctx, dmm_iters, nullptr))) return rc;
    if ((rc = dm_refine(ctx, pd_iters, nullptr))) return rc;
    if (d_u != nullptr && (rc = dm_get_disparity(ctx, d_u))) return rc;
    return DM_OK;
}

DM_API int dm_cost_volume_mirrored(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right)
{
    const Range range("dm_cost_volume_mirrored");
    int rc = ready(ctx);
    if (rc) return rc;
    if (d_left == nullptr || d_right == nullptr) return DM_ERR_ARG;
    if ((rc = census_cost(ctx, d_left, d_right, true))) return rc;
    return dm_reset_duals(ctx);
}

DM_API int dm_lr_check(const float* d_u_left, const float* d_u_mirrored, int H, int W,
                       float max_diff, uint8_t* d_ok, float* d_u_out, float* d_u_right,
                       void* stream)
{
    if (d_u_left == nullptr || d_u_mirrored == nullptr || d_ok == nullptr || d_u_out == nullptr)
        return DM_ERR_ARG;
    if (H <= 0 || W <= 0 || (long long)H * W > (1LL << 31) || !(max_diff >= 0.0f) ||
        !std::isfinite(max_diff))
        return DM_ERR_ARG;
    DM_CK(dm::launch_lr_check(d_u_left, d_u_mirrored, H, W, max_diff, d_ok, d_u_out, d_u_right,
                              static_cast<cudaStream_t>(stream)));
    return DM_OK;
}

DM_API int dm_solve_lr(dm_ctx* left, dm_ctx* right, const uint8_t* d_left, const uint8_t* d_right,
                       int dmm_iters, int pd_iters, float max_diff, uint8_t* d_ok, float* d_u,
                       float* d_u_right)
{
    const Range range("dm_solve_lr");
    int rc;
    if ((rc = ready(left)) || (rc = ready(right))) return rc;
    if (left == right || left->H != right->H || left->W != right->W || left->L != right->L ||
        left->cost_bytes != right->cost_bytes)
        return DM_ERR_ARG;
    if (d_left == nullptr || d_right == nullptr || d_ok == nullptr || d_u == nullptr)
        return DM_ERR_ARG;
    if (!(max_diff >= 0.0f) || !std::isfinite(max_diff)) return DM_ERR_ARG;
    const bool fork = left->stream != right->stream;
    if (fork) {
        if (left->ev_fork == nullptr)
            DM_CK(cudaEventCreateWithFlags(&left->ev_fork, cudaEventDisableTiming));
        if (left->ev_join == nullptr)
            DM_CK(cudaEventCreateWithFlags(&left->ev_join, cudaEventDisableTiming));
        // the inputs are ready in the left stream's order
        DM_CK(cudaEventRecord(left->ev_fork, left->stream));
        DM_CK(cudaStreamWaitEvent(right->stream, left->ev_fork, 0));
    }
    // right view: the mirrored pair through the unchanged path, on its own stream
    if ((rc = dm_cost_volume_mirrored(right, d_left, d_right))) return rc;
    if ((rc = dm_discrete(right, dmm_iters, nullptr))) return rc;
    // two one-launch refinements that may overlap would each hold resident
    // CTAs at grid barriers: the forked view takes one launch per iteration
    // (the same result bit for bit)
    const int32_t pd_launch = right->p.pd_launch;
    if (fork) right->p.pd_launch = 1;
    rc = dm_refine(right, pd_iters, nullptr);
    right->p.pd_launch = pd_launch;
    if (rc) return rc;
    // left view, concurrently when the streams differ
    if ((rc = dm_solve(left, d_left, d_right, dmm_iters, pd_iters, nullptr))) return rc;
    if (fork) {
        DM_CK(cudaEventRecord(left->ev_join, right->stream));
        DM_CK(cudaStreamWaitEvent(left->stream, left->ev_join, 0));
    }
    const dm::PdArgs al = pd_args(left);
    const dm::PdArgs ar = pd_args(right);
    DM_CK(dm::launch_lr_check(al.u, ar.u, left->H, left->W, max_diff, d_ok, d_u, d_u_right,
                              left->stream));
    left->launches += 1;
    return DM_OK;
}

// ---- optical flow ----------------------------------------------------------

namespace {
// make `later` wait for the work queued on `earlier` so far (no-op on one stream)
int order_streams(dm_ctx* owner, cudaStream_t earlier, cudaStream_t later)
{
    if (earlier == later) return DM_OK;
    if (owner->ev_fork == nullptr)
        DM_CK(cudaEventCreateWithFlags(&owner->ev_fork, cudaEventDisableTiming));
    DM_CK(cudaEventRecord(owner->ev_fork, earlier));
    DM_CK(cudaStreamWaitEvent(later, owner->ev_fork, 0));
    return DM_OK;
}
}  // namespace

DM_API int dm_flow_cost_volumes(dm_ctx* layer1, dm_ctx* layer2, const uint8_t* d_img1,
                                const uint8_t* d_img2, int lo1, int lo2)
{
    const Range range("dm_flow_cost_volumes");
    int rc;
    if ((rc = ready(layer1)) || (rc = ready(layer2))) return rc;
    if (layer1 == layer2 || layer1->H != layer2->H || layer1->W != layer2->W) return DM_ERR_ARG;
    if (d_img1 == nullptr || d_img2 == nullptr) return DM_ERR_ARG;
    if (lo1 < -65535 || lo1 > 65535 || lo2 < -65535 || lo2 > 65535) return DM_ERR_ARG;
    if (layer1->p.census_win != layer2->p.census_win) return DM_ERR_ARG;
    if (layer1->cost_bytes != 1 || layer2->cost_bytes != 1) return DM_ERR_STATE;
    const int H = layer1->H, W = layer1->W;
    const size_t HW = (size_t)H * W;
    const int maxc = layer1->p.census_win * layer1->p.census_win - 1;
    uint32_t* census = reinterpret_cast<uint32_t*>(layer1->ws + layer1->lay.census);
    cudaStream_t s1 = layer1->stream;
    DM_CK(dm::launch_census_edges(d_img1, d_img2, H, W, layer1->p.census_win,
                                  layer1->p.edge_threshold, layer1->p.w_hi, layer1->p.w_lo, census,
                                  layer1->ws + layer1->lay.wh, layer1->ws + layer1->lay.wv, false,
                                  s1));
    DM_CK(dm::launch_flow_cost(census, census + HW, H, W, lo1, layer1->L, lo2, layer2->L, maxc,
                               layer1->ws + layer1->lay.cost, layer2->ws + layer2->lay.cost, s1));
    DM_CK(cudaMemcpyAsync(layer2->ws + layer2->lay.wh, layer1->ws + layer1->lay.wh, HW,
                          cudaMemcpyDeviceToDevice, s1));
    DM_CK(cudaMemcpyAsync(layer2->ws + layer2->lay.wv, layer1->ws + layer1->lay.wv, HW,
                          cudaMemcpyDeviceToDevice, s1));
    layer1->launches += 2;
    if ((rc = order_streams(layer1, s1, layer2->stream))) return rc;
    for (dm_ctx* c : {layer1, layer2}) {
        c->have_cost = c->have_weights = true;
        c->cost_f32 = nullptr;
        c->tape_valid = false;
        if ((rc = choose_path(c, maxc, false))) return rc;
        if ((rc = dm_reset_duals(c))) return rc;
    }
    layer1->flow_partner = layer2;
    layer1->flow_lo1 = lo1;
    layer1->flow_lo2 = lo2;
    return DM_OK;
}

DM_API int dm_flow_refine_bytes(int H, int W, size_t* bytes)
{
    if (bytes == nullptr || H <= 0 || W <= 0) return DM_ERR_ARG;
    *bytes = (size_t)dm::kFlowArrays * align_up((size_t)H * W * sizeof(float), 256);
    return DM_OK;
}

DM_API int dm_flow_refine(dm_ctx* layer1, dm_ctx* layer2, int iters, void* d_scratch,
                          size_t bytes, float* d_u1, float* d_u2)
{
    const Range range("dm_flow_refine");
    int rc;
    if ((rc = ready(layer1)) || (rc = ready(layer2))) return rc;
    if (layer1->flow_partner != layer2) return DM_ERR_STATE;
    if (!layer1->have_labels || !layer2->have_labels) return DM_ERR_STATE;
    if (iters < 0 || d_scratch == nullptr || d_u1 == nullptr || d_u2 == nullptr) return DM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(d_scratch) & 255) != 0) return DM_ERR_WORKSPACE;
    size_t need = 0;
    dm_flow_refine_bytes(layer1->H, layer1->W, &need);
    if (bytes < need) return DM_ERR_WORKSPACE;
    const dm_params& p = layer1->p;
    if (p.warps <= 0) return DM_ERR_ARG;
    const int H = layer1->H, W = layer1->W;
    const size_t HW = (size_t)H * W;
    const size_t stride = align_up(HW * sizeof(float), 256);
    dm::FlowArgs a{};
    a.H = H;
    a.W = W;
    a.lo1 = layer1->flow_lo1;
    a.K1 = layer1->L;
    a.lo2 = layer1->flow_lo2;
    a.K2 = layer2->L;
    a.maxc = p.census_win * p.census_win - 1;
    const uint32_t* census = reinterpret_cast<const uint32_t*>(layer1->ws + layer1->lay.census);
    a.c1 = census;
    a.c2 = census + HW;
    a.wh = layer1->ws + layer1->lay.wh;
    a.wv = layer1->ws + layer1->lay.wv;
    a.alpha = (float)p.alpha;
    a.lambda_r = (float)p.lambda_r;
    a.tau = (float)p.tau;
    a.sigma = (float)p.sigma;
    a.h = (float)p.h;
    a.ap = (float)p.eps;
    a.bp = (float)p.delta;
    a.bq = (float)(p.C + p.delta - p.eps * p.delta);
    float* arr[dm::kFlowArrays];
    for (int k = 0; k < dm::kFlowArrays; ++k)
        arr[k] = reinterpret_cast<float*>(static_cast<uint8_t*>(d_scratch) + k * stride);
    float** f[dm::kFlowArrays] = {&a.u1,  &a.u2,  &a.un1, &a.un2, &a.u01, &a.u02,
                                  &a.L1,  &a.L2,  &a.q11, &a.q12, &a.q22, &a.b1lo,
                                  &a.b1hi, &a.b2lo, &a.b2hi, &a.ph1, &a.pv1, &a.qh1,
                                  &a.qv1, &a.ph2, &a.pv2, &a.qh2, &a.qv2};
    for (int k = 0; k < dm::kFlowArrays; ++k) *f[k] = arr[k];
    cudaStream_t s = layer1->stream;
    if ((rc = order_streams(layer1, layer2->stream, s))) return rc;   // layer 2's labels
    DM_CK(dm::launch_flow_init(a, reinterpret_cast<const uint16_t*>(layer1->ws + layer1->lay.labels),
                               reinterpret_cast<const uint16_t*>(layer2->ws + layer2->lay.labels),
                               s));
    layer1->launches += 1;
    const int base = iters / p.warps, extra = iters % p.warps;
    for (int w = 0; w < p.warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        DM_CK(dm::launch_flow_lin(a, s));
        layer1->launches += 1;
        for (int it = 0; it < nit; ++it) {
            DM_CK(dm::launch_flow_iter(a, s));
            layer1->launches += 2;
            std::swap(a.u1, a.un1);
            std::swap(a.u2, a.un2);
        }
    }
    DM_CK(dm::launch_flow_export(a, d_u1, d_u2, s));
    layer1->launches += 1;
    return DM_OK;
}

DM_API int dm_solve_host(dm_ctx* ctx, const uint8_t* h_left, const uint8_t* h_right,
                         int dmm_iters, int pd_iters, float* h_u, uint16_t* h_labels)
{
    int rc = ready(ctx);
    if (rc) return rc;
    if (h_left == nullptr || h_right == nullptr || h_u == nullptr) return DM_ERR_ARG;
    const size_t HW = (size_t)ctx->H * ctx->W;
    uint8_t* dimg = ctx->ws + ctx->lay.img;
    DM_CK(cudaMemcpyAsync(dimg, h_left, HW, cudaMemcpyHostToDevice, ctx->stream));
    DM_CK(cudaMemcpyAsync(dimg + HW, h_right, HW, cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = dm_solve(ctx, dimg, dimg + HW, dmm_iters, pd_iters, nullptr))) return rc;
    dm::PdArgs a = pd_args(ctx);
    DM_CK(cudaMemcpyAsync(h_u, a.u, HW * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    if (h_labels != nullptr)
        DM_CK(cudaMemcpyAsync(h_labels, ctx->ws + ctx->lay.labels, HW * sizeof(uint16_t),
                              cudaMemcpyDeviceToHost, ctx->stream));
    return check_device_error(ctx);
}

DM_API int dm_set_minorant(dm_ctx* ctx, int kind, int max_pass, int gamma_num, int gamma_den)
{
    if (ctx == nullptr || kind < DM_MINORANT_HIER || kind > DM_MINORANT_ITERATIVE) return DM_ERR_ARG;
    if (kind == DM_MINORANT_ITERATIVE &&
        (max_pass < 1 || max_pass > 64 || gamma_den < 1 || gamma_den > 1024 || gamma_num < 0 ||
         gamma_num > gamma_den))
        return DM_ERR_ARG;
    ctx->minorant = kind;
    if (kind == DM_MINORANT_ITERATIVE) {
        ctx->max_pass = max_pass;
        ctx->gamma_num = gamma_num;
        ctx->gamma_den = gamma_den;
    }
    if (ctx->ws == nullptr || !ctx->have_cost) return DM_OK;
    // the dual storage follows the kernel: choose it again and start cold
    set_path(ctx, ctx->cost_max, ctx->user_weights);
    return dm_reset_duals(ctx);
}

DM_API int dm_get_path(const dm_ctx* ctx, int* kernel, int* delta_bytes)
{
    if (ctx == nullptr || kernel == nullptr || delta_bytes == nullptr) return DM_ERR_ARG;
    *kernel = ctx->use16 ? (ctx->use_g ? 8 : 16) : 32;
    *delta_bytes = ctx->use16 ? ctx->delta_bytes : 4;
    return DM_OK;
}

DM_API int dm_launch_count(const dm_ctx* ctx, uint64_t* count)
{
    if (ctx == nullptr || count == nullptr) return DM_ERR_ARG;
    *count = ctx->launches;
    return DM_OK;
}

DM_API int dm_sync(dm_ctx* ctx)
{
    int rc = ready(ctx);
    if (rc) return rc;
    return check_device_error(ctx);
}

DM_API const char* dm_error_string(int status)
{
    switch (status) {
        case DM_OK: return "ok";
        case DM_ERR_ARG: return "invalid argument";
        case DM_ERR_CUDA: return "CUDA runtime error";
        case DM_ERR_RANGE: return "value out of range for its storage type";
        case DM_ERR_TIMEOUT: return "bounded device wait timed out";
        case DM_ERR_STATE: return "invalid call order or missing workspace";
        case DM_ERR_WORKSPACE: return "workspace too small or misaligned";
        case DM_ERR_DEVICE: return "a kernel flagged invalid input data";
        default: return "unknown status";
    }
}

}  // extern "C"
