// Batched form of the hot path: many stereo pairs of mixed sizes and label
// counts solved together (declared in include/dm.h, dm_batch_*).
//
// Every pair keeps its own dm_ctx (its layout, taps and dual storage) on a
// slice of one workspace; the batch adds device tables so that the costly
// steps run as persistent kernels over all pairs at once:
//   * Dual MM passes: one launch per label class (kernel instantiation: the
//     lane-group kernel where a pair's bounds admit it, else the one-warp
//     16-bit kernel) and pass; each CTA pulls (pair, chain) tasks, longest
//     chains first, from a work counter.  Pairs outside the packed kernels'
//     bounds keep their own launches.
//   * primal-dual iterations: one launch per iteration for all pairs; the CTAs
//     stride over the tiles of every pair (tile shape from the autotuner).
// Pairs are solved in groups whose working set fits a budget (GB300's L2 holds
// 129 MB): a group runs all its Dual MM iterations and its refinement before
// the next group starts, so that each pass reads what the previous one wrote
// from L2 rather than HBM.
// dm_batch_capture records one whole solve (cost volumes, discrete and
// continuous stages, outputs) into a CUDA graph that dm_batch_replay launches.
// dm_batch_tune times the candidate launch shapes and group budgets on the
// batch itself and keeps the fastest, optionally through a cache file.

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dm_ctx.cuh"

namespace {

constexpr int kMaxBatchIters = 256;   // Dual MM iterations of one batched solve
constexpr int kMaxClasses = 24;       // kernel instantiations: (G or NP, padded, delta bytes)
constexpr int kTuning = 5;            // values of a launch-shape choice

#define DB_CK(call)                                  \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return DM_ERR_CUDA;   \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// a kernel instantiation: the lane-group kernel with g lanes per group, or
// (g = 0) the one-warp 16-bit kernel with np label pairs per lane
struct Class {
    int g = 0, np = 1, pad = 0, dbytes = 1;
};

// one persistent launch: up to kBatchDescs pairs of one class and their tasks
struct Unit {
    int cls = 0;
    std::vector<int> pairs;
    int begin = 0, count = 0;  // range in the task table
};

// a run of pairs [first, first + n) solved together, with its launches per
// pass and the offsets of its primal-dual tables
struct Group {
    int first = 0, n = 0;
    std::vector<Unit> units[2];
    int tiles_at = 0, px_at = 0;          // offsets into the prefix tables
    int total_tiles = 0;
    long long total_px = 0;
};

}  // namespace

struct dm_batch {
    int n = 0;
    std::vector<dm_ctx*> ctx;
    std::vector<size_t> ctx_off;
    dm_params p{};
    uint8_t* ws = nullptr;
    size_t total = 0;
    cudaStream_t stream = nullptr;
    int sms = 1;
    // launch shapes (from dm_batch_tune or dm_batch_set_tuning); group_mb: the
    // budget of a group's working set in MB (0: one group)
    int dmm_occ = 3, pd_tx = 32, pd_ty = 8, pd_gm = 4, group_mb = 128;
    // device tables: offsets into ws
    size_t off_tasks = 0, off_pd = 0, off_tiles = 0, off_px = 0, off_labels = 0;
    size_t off_counters = 0;
    int task_cap = 0;
    // host plan (valid after prepare)
    std::vector<Class> classes;
    std::vector<int> cls_of;    // class of each pair, -1: its own launches
    std::vector<dm::Dmm16Args> d16;  // [2 n]: pass arguments of each pair
    dm::Batch16Args launch_args{};   // assembled per launch (the launch copies it)
    std::vector<Group> groups;
    bool prepared = false;
    int prep_tx = 0, prep_ty = 0, prep_mb = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0, graph_launches = 0;
};

namespace {

int grid_1d(const dm_batch* b) { return b->sms * 8; }

// bytes a pair's two passes touch per iteration: both dual arrays and the cost
size_t pair_bytes(const dm_ctx* c)
{
    const size_t hwl = (size_t)c->H * c->W * c->L;
    const size_t per = c->use16 ? 2 * (size_t)c->delta_bytes + c->cost_bytes : 8 + c->cost_bytes;
    return hwl * per;
}

// host plan and device tables for the current launch shapes
int prepare(dm_batch* b)
{
    const int n = b->n;
    std::vector<dm::Dmm16Args>& d16 = b->d16;
    d16.assign(2 * n, dm::Dmm16Args{});
    std::vector<dm::PdArgs> pd(2 * n);
    std::vector<const uint16_t*> labels(n);
    b->classes.clear();
    b->groups.clear();
    b->cls_of.assign(n, -1);
    for (int i = 0; i < n; ++i) {
        dm_ctx* c = b->ctx[i];
        dm::ctxops::predict_path(c, c->p.census_win * c->p.census_win - 1);
        uint16_t* lab = reinterpret_cast<uint16_t*>(c->ws + c->lay.labels);
        long long* lb = reinterpret_cast<long long*>(c->ws + c->lay.lb);
        for (int w = 0; w < 2; ++w) {
            d16[w * n + i] = dm::ctxops::dm16_args(c, w);
            d16[w * n + i].labels = lab;  // used on the last vertical pass
            d16[w * n + i].lb = lb;       // + the iteration, on vertical passes
        }
        for (int par = 0; par < 2; ++par) {
            c->u_cur = c->pq_cur = par;
            pd[2 * i + par] = dm::ctxops::pd_args(c);
        }
        c->u_cur = c->pq_cur = 0;
        labels[i] = lab;
        if (!c->use16 || !c->discrete_ok) continue;
        Class want;
        want.g = c->use_g ? c->gsz : 0;
        want.np = c->use_g ? 0 : c->np16;
        want.pad = !c->use_g && c->L != 64 * c->np16 ? 1 : 0;
        want.dbytes = c->delta_bytes;
        int k = 0;
        for (; k < (int)b->classes.size(); ++k) {
            const Class& q = b->classes[k];
            if (q.g == want.g && q.np == want.np && q.pad == want.pad && q.dbytes == want.dbytes)
                break;
        }
        if (k == (int)b->classes.size()) {
            if (k == kMaxClasses) return DM_ERR_ARG;
            b->classes.push_back(want);
        }
        b->cls_of[i] = k;
    }
    // groups: consecutive pairs while their working set stays within the budget
    const size_t budget = b->group_mb > 0 ? (size_t)b->group_mb << 20 : ~(size_t)0;
    for (int i = 0; i < n;) {
        Group g;
        g.first = i;
        size_t bytes = 0;
        do {
            bytes += pair_bytes(b->ctx[i]);
            ++i;
        } while (i < n && bytes + pair_bytes(b->ctx[i]) <= budget);
        g.n = i - g.first;
        b->groups.push_back(g);
    }
    // per group: tasks (per pass, the classes one after another, longest chains
    // first) and the tile / pixel prefix tables
    const int nc = (int)b->classes.size();
    std::vector<int2> tasks;
    std::vector<int> tiles;
    std::vector<long long> px;
    for (Group& g : b->groups) {
        for (int w = 0; w < 2; ++w) {
            g.units[w].clear();
            for (int k = 0; k < nc; ++k) {
                std::vector<int> members;
                for (int i = g.first; i < g.first + g.n; ++i)
                    if (b->cls_of[i] == k) members.push_back(i);
                for (size_t at = 0; at < members.size(); at += dm::kBatchDescs) {
                    Unit u;
                    u.cls = k;
                    u.pairs.assign(members.begin() + at,
                                   members.begin() + std::min(members.size(), at + dm::kBatchDescs));
                    u.begin = (int)tasks.size();
                    for (int j = 0; j < (int)u.pairs.size(); ++j) {
                        const dm_ctx* c = b->ctx[u.pairs[j]];
                        const int chains = w == 0 ? c->H : c->W;
                        for (int ch = 0; ch < chains; ++ch) tasks.push_back(make_int2(j, ch));
                    }
                    std::stable_sort(tasks.begin() + u.begin, tasks.end(),
                                     [&](const int2& a, const int2& q) {
                                         const dm_ctx* ca = b->ctx[u.pairs[a.x]];
                                         const dm_ctx* cq = b->ctx[u.pairs[q.x]];
                                         return (w == 0 ? ca->W : ca->H) > (w == 0 ? cq->W : cq->H);
                                     });
                    u.count = (int)tasks.size() - u.begin;
                    g.units[w].push_back(u);
                }
            }
        }
        g.tiles_at = (int)tiles.size();
        g.px_at = (int)px.size();
        int t = 0;
        long long q = 0;
        for (int i = g.first; i < g.first + g.n; ++i) {
            const dm_ctx* c = b->ctx[i];
            tiles.push_back(t);
            px.push_back(q);
            t += ((c->W + b->pd_tx - 1) / b->pd_tx) * ((c->H + b->pd_ty - 1) / b->pd_ty);
            q += (long long)c->H * c->W;
        }
        tiles.push_back(t);
        px.push_back(q);
        g.total_tiles = t;
        g.total_px = q;
    }
    if ((int)tasks.size() > b->task_cap || (int)tiles.size() > 2 * n) return DM_ERR_ARG;
    uint8_t* ws = b->ws;
    if (!tasks.empty())
        DB_CK(cudaMemcpyAsync(ws + b->off_tasks, tasks.data(), tasks.size() * sizeof(int2),
                              cudaMemcpyHostToDevice, b->stream));
    DB_CK(cudaMemcpyAsync(ws + b->off_pd, pd.data(), pd.size() * sizeof(dm::PdArgs),
                          cudaMemcpyHostToDevice, b->stream));
    DB_CK(cudaMemcpyAsync(ws + b->off_tiles, tiles.data(), tiles.size() * sizeof(int),
                          cudaMemcpyHostToDevice, b->stream));
    DB_CK(cudaMemcpyAsync(ws + b->off_px, px.data(), px.size() * sizeof(long long),
                          cudaMemcpyHostToDevice, b->stream));
    DB_CK(cudaMemcpyAsync(ws + b->off_labels, labels.data(), labels.size() * sizeof(void*),
                          cudaMemcpyHostToDevice, b->stream));
    DB_CK(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
    b->prepared = true;
    b->prep_tx = b->pd_tx;
    b->prep_ty = b->pd_ty;
    b->prep_mb = b->group_mb;
    return DM_OK;
}

dm::PdBatchArgs pd_batch_args(const dm_batch* b, const Group& g, int parity)
{
    dm::PdBatchArgs a{};
    a.descs = reinterpret_cast<const dm::PdArgs*>(b->ws + b->off_pd) + 2 * g.first;
    a.tile_start = reinterpret_cast<const int*>(b->ws + b->off_tiles) + g.tiles_at;
    a.px_start = reinterpret_cast<const long long*>(b->ws + b->off_px) + g.px_at;
    a.labels = reinterpret_cast<const uint16_t* const*>(b->ws + b->off_labels) + g.first;
    a.n = g.n;
    a.total_tiles = g.total_tiles;
    a.total_px = g.total_px;
    a.parity = parity;
    return a;
}

// one batched Dual MM pass over a group: every class (+ the pairs with their
// own kernel)
int batch_pass(dm_batch* b, const Group& g, int which, int t, bool last)
{
    int* counter = reinterpret_cast<int*>(b->ws + b->off_counters);
    dm::Batch16Args& a = b->launch_args;
    for (const Unit& u : g.units[which]) {
        if (u.count == 0) continue;
        const Class& q = b->classes[u.cls];
        a.tasks = reinterpret_cast<const int2*>(b->ws + b->off_tasks) + u.begin;
        a.n_tasks = u.count;
        a.counter = counter;
        // persistent CTAs: for the one-warp kernel 256 labels (NP = 4) fit two
        // per SM, the others three; the lane-group kernel fits 24 warps per SM
        // (dmm_occ = 3 takes them all)
        int occ = q.np == 4 ? std::min(b->dmm_occ, 2) : b->dmm_occ;
        if (q.g > 0) occ = std::max(1, 8 * b->dmm_occ / std::min(q.g, 8));
        a.grid = std::min(b->sms * occ, u.count);
        a.n_desc = (int)u.pairs.size();
        for (int j = 0; j < a.n_desc; ++j) {
            dm::Dmm16Args d = b->d16[which * b->n + u.pairs[j]];
            if (which == 0 || !last) d.labels = nullptr;
            d.lb = which == 1 ? d.lb + t : nullptr;
            a.descs[j] = d;
        }
        DB_CK(cudaMemsetAsync(counter, 0, sizeof(int), b->stream));
        if (q.g > 0)
            DB_CK(dm::launch_dmg_batch(a, q.g, b->ctx[0]->radius, q.dbytes, b->stream));
        else
            DB_CK(dm::launch_dmm16_batch(a, q.np, b->ctx[0]->radius, q.pad != 0, q.dbytes,
                                         b->stream));
        b->launches += 1;
    }
    for (int i = g.first; i < g.first + g.n; ++i) {
        if (b->cls_of[i] >= 0) continue;
        dm_ctx* c = b->ctx[i];
        long long* lb = reinterpret_cast<long long*>(c->ws + c->lay.lb);
        uint16_t* lab = reinterpret_cast<uint16_t*>(c->ws + c->lay.labels);
        const unsigned long long before = c->launches;
        int rc = dm::ctxops::run_pass(c, which, (which == 1 && last) ? lab : nullptr,
                                      which == 1 ? lb + t : nullptr);
        if (rc) return rc;
        b->launches += c->launches - before;
    }
    return DM_OK;
}

int batch_pd(dm_batch* b, const Group& g, int iters)
{
    const int g1 = grid_1d(b);
    DB_CK(dm::launch_init_batch(pd_batch_args(b, g, 0), g1, b->stream));
    b->launches += 1;
    int parity = 0;
    const int warps = b->p.warps, base = iters / warps, extra = iters % warps;
    for (int w = 0; w < warps; ++w) {
        const int nit = base + (w < extra ? 1 : 0);
        if (nit == 0) continue;
        DB_CK(dm::launch_lin_batch(pd_batch_args(b, g, parity), g1, b->stream));
        b->launches += 1;
        for (int it = 0; it < nit; ++it) {
            const int grid = std::min(b->sms * b->pd_gm, std::max(1, g.total_tiles));
            DB_CK(dm::launch_pd_batch(pd_batch_args(b, g, parity), b->pd_tx, b->pd_ty, grid,
                                      b->stream));
            b->launches += 1;
            parity ^= 1;
        }
    }
    for (int i = g.first; i < g.first + g.n; ++i) {
        b->ctx[i]->u_cur = b->ctx[i]->pq_cur = parity;
        b->ctx[i]->have_u = true;
    }
    return DM_OK;
}

int batch_solve(dm_batch* b, const uint8_t* const* d_left, const uint8_t* const* d_right,
                int dmm_iters, int pd_iters, float* const* d_u)
{
    nvtxRangePushA("dm_batch_solve");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    int rc;
    const unsigned long long l0 = b->launches;
    for (int i = 0; i < b->n; ++i) {
        dm_ctx* c = b->ctx[i];
        const unsigned long long before = c->launches;
        if ((rc = dm_cost_volume(c, d_left[i], d_right[i]))) return rc;
        b->launches += c->launches - before;
        if ((c->use16 && c->discrete_ok) != (b->cls_of[i] >= 0) ||
            (b->cls_of[i] >= 0 && b->classes[b->cls_of[i]].g != (c->use_g ? c->gsz : 0)))
            return DM_ERR_STATE;  // the plan no longer matches the pair's kernel
        DB_CK(cudaMemsetAsync(c->ws + c->lay.lb, 0, dmm_iters * sizeof(long long), b->stream));
    }
    for (const Group& g : b->groups) {
        for (int t = 0; t < dmm_iters; ++t)
            for (int which = 0; which < 2; ++which)
                if ((rc = batch_pass(b, g, which, t, t == dmm_iters - 1))) return rc;
        for (int i = g.first; i < g.first + g.n; ++i) {
            b->ctx[i]->have_labels = true;
            b->ctx[i]->last_iters = dmm_iters;
        }
        if ((rc = batch_pd(b, g, pd_iters))) return rc;
    }
    if (d_u != nullptr)
        for (int i = 0; i < b->n; ++i)
            if (d_u[i] != nullptr && (rc = dm_get_disparity(b->ctx[i], d_u[i]))) return rc;
    b->graph_launches = b->launches - l0;
    return DM_OK;
}

int check_args(const dm_batch* b, const uint8_t* const* l, const uint8_t* const* r, int dmm_iters,
               int pd_iters)
{
    if (b == nullptr || l == nullptr || r == nullptr) return DM_ERR_ARG;
    if (dmm_iters < 1 || dmm_iters > kMaxBatchIters || pd_iters < 0) return DM_ERR_ARG;
    for (int i = 0; i < b->n; ++i)
        if (l[i] == nullptr || r[i] == nullptr) return DM_ERR_ARG;
    if (b->ws == nullptr) return DM_ERR_STATE;
    return DM_OK;
}

void drop_graph(dm_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// ---- autotuner -------------------------------------------------------------

float time_ms(dm_batch* b, int reps, int (*body)(dm_batch*, void*), void* arg, int* rc)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    *rc = body(b, arg);  // warm-up
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps && *rc == DM_OK; ++r) *rc = body(b, arg);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

struct SolveArgs {
    const uint8_t* const* l;
    const uint8_t* const* r;
    int dmm_iters, pd_iters;
};

int body_solve(dm_batch* b, void* arg)
{
    const SolveArgs* a = static_cast<const SolveArgs*>(arg);
    return batch_solve(b, a->l, a->r, a->dmm_iters, a->pd_iters, nullptr);
}

int body_pd(dm_batch* b, void* arg)
{
    const int iters = *static_cast<int*>(arg);
    for (const Group& g : b->groups)
        for (int it = 0; it < iters; ++it) {
            const int grid = std::min(b->sms * b->pd_gm, std::max(1, g.total_tiles));
            DB_CK(dm::launch_pd_batch(pd_batch_args(b, g, it & 1), b->pd_tx, b->pd_ty, grid,
                                      b->stream));
        }
    return DM_OK;
}

std::string tune_key(const dm_batch* b)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string k = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount);
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the shapes and the penalty
    auto mix = [&](long long v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (unsigned long long)((v >> (8 * i)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    for (const dm_ctx* c : b->ctx) {
        mix(c->H);
        mix(c->W);
        mix(c->L);
    }
    mix(b->p.w_hi);
    mix(b->p.w_lo);
    mix((long long)(b->p.C * 1000));
    char buf[32];
    std::snprintf(buf, sizeof(buf), "/%016llx", h);
    for (char& ch : k)
        if (ch == ' ') ch = '_';
    return k + buf;
}

bool read_cache(const char* path, const std::string& key, int* v)
{
    if (path == nullptr) return false;
    FILE* f = std::fopen(path, "r");
    if (f == nullptr) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[400];
        int a[kTuning];
        if (std::sscanf(line, "%399s %d %d %d %d %d", k, &a[0], &a[1], &a[2], &a[3], &a[4]) ==
                1 + kTuning &&
            key == k) {
            std::memcpy(v, a, sizeof(a));
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void write_cache(const char* path, const std::string& key, const int* v)
{
    if (path == nullptr) return;
    FILE* f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3], v[4]);
    std::fclose(f);
}

bool valid_tuning(const int* v)
{
    return v[0] >= 1 && v[0] <= 3 && dm::pd_tile_supported(v[1], v[2]) && v[3] >= 1 && v[3] <= 64 &&
           v[4] >= 0 && v[4] <= (1 << 20);
}

}  // namespace

extern "C" {

DM_API int dm_batch_create(int n, const int* H, const int* W, const int* L, const dm_params* p,
                           dm_batch** out)
{
    if (out == nullptr || p == nullptr || H == nullptr || W == nullptr || L == nullptr)
        return DM_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 4096) return DM_ERR_ARG;
    dm_batch* b = new (std::nothrow) dm_batch();
    if (b == nullptr) return DM_ERR_ARG;
    b->n = n;
    b->p = *p;
    size_t off = 0;
    int task_cap = 0;
    for (int i = 0; i < n; ++i) {
        dm_ctx* c = nullptr;
        int rc = dm_create(H[i], W[i], L[i], p, &c);
        if (rc) {
            dm_batch_destroy(b);
            return rc;
        }
        b->ctx.push_back(c);
        size_t bytes = 0;
        dm_workspace_bytes(c, &bytes);
        b->ctx_off.push_back(off);
        off = align_up(off + bytes, 256);
        task_cap += H[i] + W[i];
    }
    b->task_cap = task_cap;
    auto add = [&](size_t bytes) {
        const size_t o = align_up(off, 256);
        off = o + bytes;
        return o;
    };
    b->off_tasks = add((size_t)task_cap * sizeof(int2));
    b->off_pd = add(2 * (size_t)n * sizeof(dm::PdArgs));
    b->off_tiles = add((size_t)2 * n * sizeof(int));        // n + groups entries
    b->off_px = add((size_t)2 * n * sizeof(long long));
    b->off_labels = add((size_t)n * sizeof(void*));
    b->off_counters = add(256);
    b->total = align_up(off, 256);
    *out = b;
    return DM_OK;
}

DM_API int dm_batch_destroy(dm_batch* b)
{
    if (b == nullptr) return DM_OK;
    drop_graph(b);
    for (dm_ctx* c : b->ctx) dm_destroy(c);
    delete b;
    return DM_OK;
}

DM_API int dm_batch_workspace_bytes(const dm_batch* b, size_t* bytes)
{
    if (b == nullptr || bytes == nullptr) return DM_ERR_ARG;
    *bytes = b->total;
    return DM_OK;
}

DM_API int dm_batch_set_stream(dm_batch* b, void* stream)
{
    if (b == nullptr) return DM_ERR_ARG;
    b->stream = static_cast<cudaStream_t>(stream);
    for (dm_ctx* c : b->ctx) dm_set_stream(c, stream);
    drop_graph(b);
    return DM_OK;
}

DM_API int dm_batch_bind_workspace(dm_batch* b, void* d_workspace, size_t bytes)
{
    if (b == nullptr || d_workspace == nullptr) return DM_ERR_ARG;
    if (bytes < b->total || (reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0)
        return DM_ERR_WORKSPACE;
    b->ws = static_cast<uint8_t*>(d_workspace);
    int dev = 0;
    DB_CK(cudaGetDevice(&dev));
    DB_CK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    for (int i = 0; i < b->n; ++i) {
        size_t need = 0;
        dm_workspace_bytes(b->ctx[i], &need);
        int rc = dm_bind_workspace(b->ctx[i], b->ws + b->ctx_off[i], need);
        if (rc) return rc;
    }
    b->prepared = false;
    drop_graph(b);
    return DM_OK;
}

DM_API int dm_batch_context(dm_batch* b, int i, dm_ctx** out)
{
    if (b == nullptr || out == nullptr || i < 0 || i >= b->n) return DM_ERR_ARG;
    *out = b->ctx[i];
    return DM_OK;
}

DM_API int dm_batch_set_tuning(dm_batch* b, const int* choice)
{
    if (b == nullptr || choice == nullptr) return DM_ERR_ARG;
    if (!valid_tuning(choice)) return DM_ERR_ARG;
    b->dmm_occ = choice[0];
    b->pd_tx = choice[1];
    b->pd_ty = choice[2];
    b->pd_gm = choice[3];
    b->group_mb = choice[4];
    b->prepared = false;
    drop_graph(b);
    return DM_OK;
}

DM_API int dm_batch_get_tuning(const dm_batch* b, int* choice)
{
    if (b == nullptr || choice == nullptr) return DM_ERR_ARG;
    choice[0] = b->dmm_occ;
    choice[1] = b->pd_tx;
    choice[2] = b->pd_ty;
    choice[3] = b->pd_gm;
    choice[4] = b->group_mb;
    return DM_OK;
}

DM_API int dm_batch_solve(dm_batch* b, const uint8_t* const* d_left, const uint8_t* const* d_right,
                          int dmm_iters, int pd_iters, float* const* d_u)
{
    int rc = check_args(b, d_left, d_right, dmm_iters, pd_iters);
    if (rc) return rc;
    if (!b->prepared || b->prep_tx != b->pd_tx || b->prep_ty != b->pd_ty ||
        b->prep_mb != b->group_mb)
        if ((rc = prepare(b))) return rc;
    return batch_solve(b, d_left, d_right, dmm_iters, pd_iters, d_u);
}

DM_API int dm_batch_capture(dm_batch* b, const uint8_t* const* d_left,
                            const uint8_t* const* d_right, int dmm_iters, int pd_iters,
                            float* const* d_u)
{
    int rc = check_args(b, d_left, d_right, dmm_iters, pd_iters);
    if (rc) return rc;
    if (b->stream == nullptr) return DM_ERR_STATE;  // the legacy stream cannot be captured
    if ((rc = prepare(b))) return rc;
    drop_graph(b);
    DB_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    rc = batch_solve(b, d_left, d_right, dmm_iters, pd_iters, d_u);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != DM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != DM_OK ? rc : DM_ERR_CUDA;
    }
    b->graph = g;
    DB_CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return DM_OK;
}

DM_API int dm_batch_replay(dm_batch* b)
{
    if (b == nullptr) return DM_ERR_ARG;
    if (b->exec == nullptr) return DM_ERR_STATE;
    DB_CK(cudaGraphLaunch(b->exec, b->stream));
    b->launches += b->graph_launches;
    return DM_OK;
}

DM_API int dm_batch_sync(dm_batch* b)
{
    if (b == nullptr) return DM_ERR_ARG;
    DB_CK(cudaStreamSynchronize(b->stream));
    for (dm_ctx* c : b->ctx) {
        int rc = dm_sync(c);
        if (rc) return rc;
    }
    return DM_OK;
}

DM_API int dm_batch_discrete_pass(dm_batch* b, int which)
{
    if (b == nullptr || (which != 0 && which != 1)) return DM_ERR_ARG;
    if (!b->prepared || b->ws == nullptr) return DM_ERR_STATE;
    for (const Group& g : b->groups) {
        int rc = batch_pass(b, g, which, 0, false);
        if (rc) return rc;
    }
    return DM_OK;
}

DM_API int dm_batch_launch_count(const dm_batch* b, uint64_t* count)
{
    if (b == nullptr || count == nullptr) return DM_ERR_ARG;
    *count = b->launches;
    return DM_OK;
}

DM_API int dm_batch_tune(dm_batch* b, const uint8_t* const* d_left, const uint8_t* const* d_right,
                         const char* cache_path, int* choice)
{
    int rc = check_args(b, d_left, d_right, 1, 0);
    if (rc) return rc;
    const std::string key = tune_key(b);
    int v[kTuning];
    if (read_cache(cache_path, key, v) && valid_tuning(v)) {
        if ((rc = dm_batch_set_tuning(b, v))) return rc;
        if (choice) dm_batch_get_tuning(b, choice);
        return prepare(b);
    }
    drop_graph(b);
    if ((rc = prepare(b))) return rc;
    // state to time on: the cost volumes and one iteration of both stages
    if ((rc = batch_solve(b, d_left, d_right, 1, 1, nullptr))) return rc;
    // group budget and CTAs per SM of the persistent Dual MM kernels, jointly:
    // whole solves of 2 Dual MM iterations
    static const int budgets[5] = {32, 64, 128, 256, 0};
    SolveArgs sa{d_left, d_right, 2, 0};
    float best = 1e30f;
    int best_mb = b->group_mb, best_occ = b->dmm_occ;
    for (int mb : budgets) {
        b->group_mb = mb;
        if ((rc = prepare(b))) return rc;
        for (int occ = 2; occ <= 3; ++occ) {
            b->dmm_occ = occ;
            const float ms = time_ms(b, 1, body_solve, &sa, &rc);
            if (rc) return rc;
            if (ms < best) {
                best = ms;
                best_mb = mb;
                best_occ = occ;
            }
        }
    }
    b->group_mb = best_mb;
    b->dmm_occ = best_occ;
    if ((rc = prepare(b))) return rc;
    // primal-dual: tile shape and CTAs per SM of the persistent iteration kernel
    static const int shapes[6][2] = {{32, 8}, {32, 4}, {64, 4}, {32, 16}, {16, 16}, {64, 8}};
    static const int gms[3] = {2, 4, 8};
    best = 1e30f;
    int bt[3] = {b->pd_tx, b->pd_ty, b->pd_gm};
    int iters = 10;
    for (const auto& sh : shapes) {
        b->pd_tx = sh[0];
        b->pd_ty = sh[1];
        if ((rc = prepare(b))) return rc;
        for (int gm : gms) {
            b->pd_gm = gm;
            const float ms = time_ms(b, 2, body_pd, &iters, &rc);
            if (rc) return rc;
            if (ms < best) {
                best = ms;
                bt[0] = sh[0];
                bt[1] = sh[1];
                bt[2] = gm;
            }
        }
    }
    b->pd_tx = bt[0];
    b->pd_ty = bt[1];
    b->pd_gm = bt[2];
    if ((rc = prepare(b))) return rc;
    dm_batch_get_tuning(b, v);
    write_cache(cache_path, key, v);
    if (choice) std::memcpy(choice, v, sizeof(v));
    return DM_OK;
}

}  // extern "C"
