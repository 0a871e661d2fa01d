// Internal declarations shared by the CUDA translation units of libdm.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dm.h"

namespace dm {

// Penalty taps per edge weight omega (0..255): row = [T_1 .. T_RMAX, P2, valid, pad, pad].
// T_d = omega * r(d) for d = 1..RMAX (capped at P2), P2 = omega * C is the
// truncation; the sampled pairwise table is V(0) = 0, V(d) = T_d for d <= RMAX,
// V(d) = P2 beyond.
constexpr int kRMax = 4;
constexpr int kTapW = 8;
constexpr int kTapP2 = kRMax;
constexpr int kTapValid = kRMax + 1;

// A value that never wins a minimisation and cannot overflow when two of them
// and a few penalties are added in int32.
constexpr int kInf = 1 << 29;

// device-side error codes written to the workspace error word
constexpr int kDevErrBadOmega = 1;
constexpr int kDevErrRange = 2;
constexpr int kDevErrIndex = 4;  // checked builds: an index outside its array (access skipped)
constexpr int kDevErrTimeout = 8;  // a bounded device-side wait gave up

struct Layout {
    size_t cost, census, img, wh, wv, lam_h, lam_v, fmsg, bmsg, labels, lb, taps, taps16;
    size_t u, u_new, u0, s1, s2, lo, hi, ph, pv, qh, qv, ph2, pv2, qh2, qv2, epart, err, bar, pool;
    size_t total;
};

struct DmmArgs {
    int which;              // 0 horizontal chains (rows), 1 vertical chains (columns)
    int H, W, L, KP;        // KP: labels padded to 32 * LPT
    const uint8_t* cost;    // [H][W][L] uint8, or
    const uint16_t* cost16; // [H][W][L] uint16 when not null
    const int32_t* lam_in;  // lambda_v (which = 0) or lambda_h (which = 1)
    int32_t* lam_out;       // lambda_h (which = 0) or lambda_v (which = 1)
    const uint8_t* wedge;   // wh (which = 0) or wv (which = 1)
    int32_t* fmsg;          // [chains][n][KP] scratch: messages entering from the left
    int32_t* bmsg;          // [chains][n][KP] scratch: messages entering from the right
    const int32_t* taps;    // [256][kTapW]
    int32_t* err;
    // finalisation (last vertical pass of a dm_discrete call)
    uint16_t* labels;       // nullable: per-pixel argmin of lambda_h + lambda_v
    long long* lb;          // nullable: sum_i min_l (lambda_h + lambda_v)_i(l)
    // chain minorant: 0 hierarchical (App. A), 1 naive, 2 iterative with
    // max_pass passes and gamma = gamma_num / gamma_den before the last pass
    int minorant, max_pass, gamma_num, gamma_den;
};

// Packed 16-bit Dual MM pass (dmm16.cu).  Duals are stored as an int32 base per
// pixel plus a delta vector ([H][W][L], uint8 or int16): lambda_h itself, and
// c + lambda_v (the unary of the horizontal pass) in place of lambda_v;
// messages as packed int16 pairs ([chains][n][32*NP] uint32) plus an int32
// offset ([chains][n]).
struct Dmm16Args {
    int which, H, W, L;
    const uint8_t* cost;
    const uint16_t* cost16;  // used in place of cost when not null
    const int32_t* base_in;
    const void* delta_in;
    int32_t* base_out;
    void* delta_out;
    const uint8_t* wedge;
    uint32_t* fmsg;
    uint32_t* bmsg;
    int32_t* fofs;
    int32_t* bofs;
    const uint32_t* taps16;  // [256][kTapW]: T_1..T_4 in both halves, P2, valid
    int32_t* err;
    uint16_t* labels;
    long long* lb;
    int seg_cap;             // entries of each segment-start array: 2^ceil(log2 n) + 1, padded
    // nullable: the counters of the split lane-group pass ([0] units taken,
    // [1] CTAs done); zero at launch and again after it
    int32_t* pool;
};
constexpr int kPoolHead = 8;   // ints of a pool

// Persistent batched form of the 16-bit pass over the chains of up to
// kBatchDescs pairs of one label class (dmm16_impl.cuh).  The descriptors travel
// in the kernel's parameter space, like the single-pair kernel's arguments.
constexpr int kBatchDescs = 96;
struct Batch16Args {
    const int2* tasks;       // (descriptor, chain), longest chains first
    int n_tasks;
    int* counter;            // work counter, zero at launch
    int grid;                // CTAs
    int n_desc;
    Dmm16Args descs[kBatchDescs];  // labels, lb: set for this launch (nullable)
};

struct PdArgs {
    int H, W, L;
    const uint8_t* cost;     // [H][W][L] uint8 samples, used when the others are null
    const uint16_t* cost16;  // [H][W][L] uint16 samples (nullable)
    const float* costf;      // [H][W][L] float32 samples (nullable)
    const float* alpha_px;   // [H][W] data weights (nullable: alpha)
    const uint8_t* wh;
    const uint8_t* wv;
    float alpha, lambda_r, tau, sigma, h;
    float ap, bp, bq;       // (alpha, beta) of R+, beta of R-
    float* u;
    float* u_new;
    float* u0;
    float* s1;
    float* s2;
    float* lo;
    float* hi;
    float* ph;               // p, q of the current iterate
    float* pv;
    float* qh;
    float* qv;
    float* ph2;              // p, q written by the iteration (ping-pong)
    float* pv2;
    float* qh2;
    float* qv2;
};

// The whole refinement in one cooperative launch (pd.cu): both ping-pong sets
// (set[1] is set[0] with u/u_new and p, q/p2, q2 swapped), the start, the
// iteration count and the grid barrier.
struct PdRunArgs {
    PdArgs set[2];
    const uint16_t* labels;  // nullable: u already holds the start
    int iters, warps;
    unsigned* bar;           // arrival counter, zero at launch
    int32_t* err;            // kDevErrTimeout when a barrier wait gives up
    long long wait_ns;       // bound of one barrier wait
    int bar_skew;            // arrivals that never come (0; > 0 only to test the bound)
};

// The whole refinement with the state resident in shared memory (pd.cu): the
// image is cut into nx x ny regions of RW x RH pixels, one CTA each.  A CTA
// holds its region and a K-pixel margin from its neighbours (EW x EH at most)
// and runs up to K iterations on it between exchanges; an exchange writes each
// region's K-wide border into one of the two workspace state sets (by the
// exchange's parity), passes a grid barrier and reads the margins back.
struct PdResArgs {
    PdArgs a;                // cost, weights, parameters, both state sets, u0, s1, s2
    const uint16_t* labels;  // nullable: a.u already holds the start
    int iters, warps;
    int nx, ny, RW, RH, K, EW, EH, TR;  // regions, margin, stored area, rows per thread round
    unsigned* bar;           // arrival counter, zero at launch
    int32_t* err;            // kDevErrTimeout when a barrier wait gives up
    long long wait_ns;       // bound of one barrier wait
    int wait_skew;           // arrivals that never come (0; > 0 only to test the bound)
};

// launch shape of pd_res_kernel (pd_res_plan)
struct PdResPlan {
    int nx, ny, RW, RH, K, EW, EH, TR, threads;
    int NS;                  // the kernel's array stride (>= EW * EH)
    size_t smem;
};

// the state set (0: u, ph, pv, qh, qv; 1: u_new, ph2, ...) that holds the
// result of pd_res_kernel: the parity of its number of exchanges
int pd_res_result_set(int iters, int warps, int K);

// Batched primal-dual kernels (pd.cu): two descriptors per pair (set 0 -> set 1
// and set 1 -> set 0), the first tile and the first pixel of each pair.
struct PdBatchArgs {
    const PdArgs* descs;        // [2 n]: descs[2 p + parity]
    const int* tile_start;      // [n + 1] for the launch's tile shape
    const long long* px_start;  // [n + 1]
    const uint16_t* const* labels;  // [n] device pointers (init)
    int n, total_tiles;
    long long total_px;
    int parity;
};

// Reverse of one primal-dual iteration k (pd.cu): state k (u, p, q) and
// u_{k+1} in, adjoints of the iteration's outputs in, adjoints of its inputs
// out (ping-pong), per-pixel accumulators updated in place.
struct AdjArgs {
    int H, W, L;
    const uint8_t* wh;
    const uint8_t* wv;
    float lambda_r, tau, sigma, h, ap, bp, bq;
    const float* u;          // state k
    const float* un;         // u_{k+1}
    const float* ph;
    const float* pv;
    const float* qh;
    const float* qv;
    const float* u0;         // linearisation of the warp
    const float* s1;
    const float* s2;
    const float* lo;
    const float* hi;
    const float* ub;         // adjoints of u_{k+1}, p_{k+1}, q_{k+1}
    const float* phb;
    const float* pvb;
    const float* qhb;
    const float* qvb;
    float* ub2;              // adjoints of u_k, p_k, q_k
    float* phb2;
    float* pvb2;
    float* qhb2;
    float* qvb2;
    float* gu0;              // adjoint of the linearisation point (through u0, lo, hi)
    float* gs1;              // adjoints of the slopes after the convexity fix
    float* gs2;
    float* glam;             // d loss / d lambda_r, per pixel (its two edges)
};

// Reverse of the linearisation of one warp (pd.cu)
struct LinAdjArgs {
    int H, W, L;
    const uint8_t* cost;
    const uint16_t* cost16;
    const float* costf;
    const float* alpha_px;
    float alpha, h;
    const float* u0;         // the warp's linearisation point
    float* gu0;
    float* gs1;
    float* gs2;
    float* ub;               // adjoint of u at the warp start (accumulated)
    float* gcost;            // [H][W][L] (nullable)
    float* galpha;           // [H][W] (nullable)
};

// Forward mode of one primal-dual iteration (pd.cu): the forward iteration of
// f and, on the same branches, the tangents of its outputs.
struct JvpArgs {
    PdArgs f;
    const float* du;         // tangents of u, p, q
    const float* dph;
    const float* dpv;
    const float* dqh;
    const float* dqv;
    float* du2;              // tangents written by the iteration
    float* dph2;
    float* dpv2;
    float* dqh2;
    float* dqv2;
    float* du0;              // tangents of the linearisation (written by launch_lin_jvp)
    float* ds1;
    float* ds2;
    float* dlo;
    float* dhi;
    const float* dcost;      // [H][W][L] tangent of the cost samples (nullable)
    const float* dalpha;     // [H][W] tangent of alpha (nullable)
    float dlambda;           // tangent of lambda_r
};

// dm_abi.cu: row of taps for one omega; returns the window radius or -1
int penalty_taps(int omega, int L, const dm_params& p, int32_t* row);
// dm_abi.cu: the parameter check of dm_create
bool params_valid(const dm_params& p);

// cost.cu
cudaError_t launch_census_edges(const uint8_t* left, const uint8_t* right, int H, int W, int win,
                                int T, int w_hi, int w_lo, uint32_t* census, uint8_t* wh,
                                uint8_t* wv, bool mirror, cudaStream_t s);
cudaError_t launch_cost(const uint32_t* census, int H, int W, int L, int maxc, void* cost,
                        int cost_bytes, cudaStream_t s);

// flow.cu: optical flow (decoupled costs and the two-component refinement)
struct FlowArgs {
    int H, W, lo1, K1, lo2, K2, maxc;
    const uint32_t* c1;      // census of image 1 [H][W]
    const uint32_t* c2;      // census of image 2 [H][W]
    const uint8_t* wh;
    const uint8_t* wv;
    float alpha, lambda_r, tau, sigma, h;
    float ap, bp, bq;        // (alpha, beta) of R+, beta of R-
    float* u1;               // current iterate (label coordinates)
    float* u2;
    float* un1;              // next iterate
    float* un2;
    float* u01;              // linearisation point
    float* u02;
    float* L1;               // gradient and PSD Hessian of the quadratic model
    float* L2;
    float* q11;
    float* q12;
    float* q22;
    float* b1lo;             // boxes
    float* b1hi;
    float* b2lo;
    float* b2hi;
    float* ph1;              // duals of component 1 and 2
    float* pv1;
    float* qh1;
    float* qv1;
    float* ph2;
    float* pv2;
    float* qh2;
    float* qv2;
};
constexpr int kFlowArrays = 23;  // float arrays of the refinement scratch
cudaError_t launch_flow_cost(const uint32_t* c1, const uint32_t* c2, int H, int W, int lo1, int K1,
                             int lo2, int K2, int maxc, uint8_t* p1, uint8_t* p2, cudaStream_t s);
cudaError_t launch_flow_init(const FlowArgs& a, const uint16_t* lab1, const uint16_t* lab2,
                             cudaStream_t s);
cudaError_t launch_flow_lin(const FlowArgs& a, cudaStream_t s);
cudaError_t launch_flow_iter(const FlowArgs& a, cudaStream_t s);
cudaError_t launch_flow_export(const FlowArgs& a, float* d1, float* d2, cudaStream_t s);

// lr.cu: two-sided consistency check of a left-view disparity and the
// disparity of the mirrored (right-view) problem
cudaError_t launch_lr_check(const float* ul, const float* um, int H, int W, float max_diff,
                            uint8_t* ok, float* out, float* ur, cudaStream_t s);

// dmm.cu
cudaError_t launch_dmm_pass(const DmmArgs& a, int lpt, int radius, cudaStream_t s);

// dmm16.cu
cudaError_t launch_dmm16_batch(const Batch16Args& b, int np, int radius, bool pad, int delta_bytes,
                               cudaStream_t s);
cudaError_t launch_dmm16_pass(const Dmm16Args& a, int np, int radius, int delta_bytes,
                              cudaStream_t s);
// Dual MM pass on lane groups (dmg_impl.cuh): g lanes of 16 labels per message
// (L <= 16 g), 8-bit messages at fmsg/bmsg ([chains][n][16 g] bytes) with int32
// offsets at fofs/bofs
cudaError_t launch_dmg_pass(const Dmm16Args& a, int g, int radius, int delta_bytes, cudaStream_t s);
int dmg_pass_kernels(const Dmm16Args& a, int g);
// persistent lane-group pass over the chains of many pairs of one label class (G lanes per group)
cudaError_t launch_dmg_batch(const Batch16Args& b, int g, int radius, int delta_bytes, cudaStream_t s);
cudaError_t launch_validate_edges(const uint8_t* wh, const uint8_t* wv, int H, int W,
                                  const int32_t* taps, int32_t* err, cudaStream_t s);
cudaError_t launch_duals_to_i32(const int32_t* base, const void* delta, int delta_bytes,
                                const void* cost, int cost_bytes, long long n_px, int L,
                                int32_t* out, cudaStream_t s);
cudaError_t launch_theta_h_init(const void* cost, int cost_bytes, int32_t* base, void* delta,
                                int delta_bytes, long long n_px, int L, cudaStream_t s);
cudaError_t launch_theta_h_from_i32(const int32_t* lam_v, const void* cost, int cost_bytes,
                                    int32_t* base, void* delta, int delta_bytes, long long n_px,
                                    int L, int32_t* err, cudaStream_t s);

// pd.cu
cudaError_t launch_init_u_from_labels(const uint16_t* labels, float* u, int n, cudaStream_t s);
cudaError_t launch_linearise(const PdArgs& a, cudaStream_t s);
cudaError_t launch_pd_iter(const PdArgs& a, cudaStream_t s);
cudaError_t launch_pd_run(const PdRunArgs& r, cudaStream_t s);
bool pd_res_plan(int H, int W, PdResPlan* plan);
cudaError_t launch_pd_res(const PdResArgs& r, const PdResPlan& plan, cudaStream_t s);
cudaError_t launch_pd_adjoint(const AdjArgs& a, cudaStream_t s);
bool pd_tile_supported(int tx, int ty);
cudaError_t launch_pd_batch(const PdBatchArgs& b, int tx, int ty, int grid, cudaStream_t s);
cudaError_t launch_lin_batch(const PdBatchArgs& b, int grid, cudaStream_t s);
cudaError_t launch_init_batch(const PdBatchArgs& b, int grid, cudaStream_t s);
cudaError_t launch_lin_adjoint(const LinAdjArgs& a, cudaStream_t s);
cudaError_t launch_lin_jvp(const JvpArgs& a, cudaStream_t s);
cudaError_t launch_pd_jvp(const JvpArgs& a, cudaStream_t s);
cudaError_t launch_sum_f32(const float* x, int n, double* partial, double* out, cudaStream_t s);
cudaError_t launch_zero_f32(float* p, size_t n, cudaStream_t s);
cudaError_t launch_energy(const PdArgs& a, double eps, double delta, double C, double* partial,
                          int nblocks, cudaStream_t s);
int energy_blocks(int H, int W);

}  // namespace dm
