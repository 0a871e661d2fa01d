// The context behind dm_ctx* (dm_abi.cu) and the operations on it that the
// batched runtime (dm_batch.cu) shares.

#pragma once

#include <vector>

#include "dm_internal.cuh"

struct dm_ctx {
    int H = 0, W = 0, L = 0, KP = 0, lpt = 0, radius = 1;
    bool discrete_ok = true;    // w_hi and w_lo have integer penalty taps within kRMax
    // packed 16-bit Dual MM (dmm16.cu): usable when L is a multiple of 2*np16 and
    // every penalty cap is small; delta_bytes is chosen per cost volume
    bool can16 = false;
    bool use16 = false;
    int np16 = 1;
    // the lane-group kernel (dmg_impl.cuh) is the packed kernel of choice when
    // every penalty cap fits its 8-bit messages; gsz lanes of 16 labels per message
    bool can_g = false;
    bool use_g = false;
    bool pool_g = true;         // the lane-group pass may run split (dmg_units_kernel)
    int gsz = 8;
    int delta_bytes = 2;
    int p2_all = 0;             // largest cap omega*C over every usable omega
    int p2_used = 0;            // largest cap over w_hi, w_lo
    std::vector<uint32_t> taps16;
    dm_params p{};
    dm::Layout lay{};
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    std::vector<int32_t> taps;  // [256][kTapW]
    bool have_cost = false;
    bool have_labels = false;
    bool have_u = false;
    int u_cur = 0;              // 0: current disparity in lay.u, 1: in lay.u_new
    int pq_cur = 0;             // 0: current p, q in lay.ph.., 1: in lay.ph2..
    int last_iters = 0;
    unsigned long long launches = 0;  // kernels enqueued by this context
    bool have_weights = false;  // edge weights in the workspace
    int cost_bytes = 1;         // storage of the cost volume: uint8 or uint16
    int cost_max = 0;           // bound on the current cost volume's samples
    // differentiable form: a caller's float cost volume and per-pixel data
    // weights (borrowed, nullable) and the tape of the last checkpointed forward
    const float* cost_f32 = nullptr;
    const float* alpha_px = nullptr;
    const void* tape = nullptr;
    size_t tape_bytes = 0;
    int tape_iters = 0, tape_ckpt = 0;
    bool tape_valid = false;
    // two-view solve: fork to the right view's stream and join back (created on
    // first use, destroyed by dm_destroy)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // chain minorant of the Dual MM passes (0 hierarchical; 1 naive and 2
    // iterative run on the int32 kernel)
    int minorant = 0, max_pass = 3, gamma_num = 1, gamma_den = 4;
    bool user_weights = false;  // the current edge weights came from the caller
    // optical flow: the partner layer and displacement offsets set by
    // dm_flow_cost_volumes on the first layer (its census holds both images)
    dm_ctx* flow_partner = nullptr;
    int flow_lo1 = 0, flow_lo2 = 0;
    // a captured solve (dm_capture) and its executable graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
};

namespace dm {
namespace ctxops {
PdArgs pd_args(dm_ctx* c);
// arguments of one 16-bit pass (labels, lb: the context's arrays, not set)
Dmm16Args dm16_args(dm_ctx* c, int which);
// one Dual MM pass with the context's own kernel
int run_pass(dm_ctx* c, int which, uint16_t* labels, long long* lb);
// the kernel and dual storage a census cost volume (values <= cost_max) gets
void predict_path(dm_ctx* c, int cost_max);
size_t base_bytes(const dm_ctx* c);
}  // namespace ctxops
}  // namespace dm
