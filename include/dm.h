/*
 * dm.h -- C ABI of the GB300 dense-matching library (libdm.so).
 *
 * The library computes the data-parallel hot path of the discrete-continuous
 * stereo method of arXiv 1601.06274 ("Solving Dense Image Matching in
 * Real-Time using Discrete-Continuous Optimization"):
 *
 *   1. census transform and matching-cost volume  (Sec. 3.1; Sec. 1)
 *   2. Dual MM over horizontal and vertical chains (Sec. 2.3, Alg. Dual_MM)
 *      with hierarchical minorants               (App. A, Alg. Handshake)
 *   3. non-linear primal-dual refinement           (Sec. 2.4, Eq. cont_iterates;
 *                                                   Sec. 3.1 data term and prox)
 *
 * and, around it: a batched form (many pairs, persistent kernels, one CUDA
 * graph), a differentiable form of the refinement, a streaming form (uint16
 * costs, warm start), the two-sided consistency check (Sec. 4.1.1), the naive
 * and iterative chain minorants (Sec. 2.3, App. A) and optical flow with
 * decoupled layers (Sec. 2.2 "Flow").
 *
 * Conventions shared by every entry point
 *   - Images are H x W, row-major, uint8, one byte per pixel (no padding).
 *   - The cost volume is [H][W][L] uint8 (uint16 with params.cost_bytes = 2),
 *     labels innermost; label l is the disparity l pixels (right-image pixel
 *     x - l).
 *   - Edge weights omega are [H][W] uint8: wh[y][x] belongs to the edge
 *     (y,x)-(y,x+1), wv[y][x] to (y,x)-(y+1,x); entries without an edge are
 *     ignored.
 *   - Dual variables lambda_h, lambda_v are [H][W][L] int32.
 *   - "d_" pointers are device pointers, "h_" pointers host pointers.  All
 *     device memory is owned by the caller.  The context owns host memory
 *     only; its device workspace is caller-allocated and bound with
 *     dm_bind_workspace().
 *   - Every call is asynchronous on the context's stream (default stream 0)
 *     unless stated otherwise; device outputs are valid once the stream has
 *     been synchronised.  Calls that return host data synchronise the stream.
 *   - Every entry point returns a status code (DM_OK on success).  No
 *     exception crosses the ABI.  Device-side faults detected by the kernels
 *     are recorded in the workspace and reported by the next synchronising
 *     call: DM_ERR_RANGE for a dual outside the packed storage's range,
 *     DM_ERR_DEVICE otherwise (e.g. an edge weight with no integer penalty
 *     table), DM_ERR_TIMEOUT when a bounded device-side wait gave up (the
 *     waits between the iterations of the one-launch refinements; the kernel
 *     then returns and the context stays usable, its refined disparity
 *     undefined).
 *   - The main stages open NVTX ranges named after their entry points.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef DM_H
#define DM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DM_API __attribute__((visibility("default")))
#else
#define DM_API
#endif

/* status codes */
#define DM_OK            0
#define DM_ERR_ARG       1  /* invalid argument (null pointer, size, parameter)   */
#define DM_ERR_CUDA      2  /* a CUDA runtime call failed                          */
#define DM_ERR_RANGE     3  /* a value does not fit the storage type               */
#define DM_ERR_TIMEOUT   4  /* a bounded device-side wait gave up                  */
#define DM_ERR_STATE     5  /* call order (e.g. no workspace, no cost volume yet)  */
#define DM_ERR_WORKSPACE 6  /* bound workspace too small or misaligned             */
#define DM_ERR_DEVICE    7  /* a kernel flagged invalid data                       */

/*
 * Parameters.  Defaults (dm_default_params) are the readings of the paper
 * used throughout: 5x5 census; omega = 8 if |I1(i) - I1(j)| < 16 else 4;
 * r of Eq. (r-decompose) with eps = 1/4, delta = 1, C = 2; tau = sigma =
 * 0.35; h = 1 label; 5 warps (Sec. 4.1.2 uses 5 warps).
 *
 * Discrete stage: the pairwise term of the edge ij is omega_ij * r(|x_i - x_j|)
 * with r sampled at integer label distances; every omega in 0..255 for which
 * omega*r(t) is an integer for all t is usable, and the table must reach its
 * cap omega*C within 4 label steps.
 * Continuous stage: the regulariser is lambda_r * omega_ij * r((Au)_ij).
 */
typedef struct dm_params {
    uint32_t struct_size;   /* sizeof(dm_params); checked by dm_create          */
    int32_t census_win;     /* 3 or 5                                            */
    int32_t edge_threshold; /* T of the edge-weight rule                         */
    int32_t w_hi, w_lo;     /* omega for |I(i) - I(j)| < T and otherwise         */
    double eps, delta, C;   /* penalty r (Eq. r-decompose)                       */
    double lambda_r;        /* regularisation weight of the continuous stage     */
    double alpha;           /* data-term weight of the continuous stage          */
    double tau, sigma;      /* primal and dual step sizes (Eq. cont_iterates)    */
    double h;               /* linearisation half-width in labels (Sec. 3.1)    */
    int32_t warps;          /* re-linearisations of the data term (Sec. 3.1)    */
    int32_t dmm_path;       /* Dual MM kernel: 0 = automatic (packed 16-bit     */
                            /* arithmetic on lane groups with 8-bit messages     */
                            /* whenever its value bounds hold; from 128 labels   */
                            /* on, a pass's depth-first work is shared by        */
                            /* persistent CTAs (at 128 labels, the horizontal    */
                            /* pass's only);                                     */
                            /* else one warp per chain, else int32), 1 = always  */
                            /* the int32 kernel, 2 = packed one-warp-per-chain   */
                            /* kernel where its bounds hold, else int32, 3 = as  */
                            /* 0 with one CTA per chain (no sharing).  All give  */
                            /* the same results bit for bit                      */
    int32_t cost_bytes;     /* storage of the cost volume: 0 or 1 = uint8,       */
                            /* 2 = uint16                                        */
    int32_t pd_launch;      /* dm_refine: 0 = automatic: all iterations in one   */
                            /* cooperative launch with the state in shared       */
                            /* memory, one region per SM, where it fits, else 1; */
                            /* 1 = one launch per iteration; 2 = one cooperative */
                            /* launch, state in global memory, grid barriers.    */
                            /* Same results bit for bit                          */
    int32_t wait_test;      /* diagnostics, 0 in normal use: > 0 makes the waits */
                            /* of the one-launch refinements wait for progress   */
                            /* that never comes, so each wait (bounded to 20 ms  */
                            /* in this mode, 1 s otherwise) gives up and         */
                            /* DM_ERR_TIMEOUT is reported                         */
    int32_t reserved[3];
} dm_params;

typedef struct dm_ctx dm_ctx;

/* Fill *p with the defaults.  DM_ERR_ARG if p is NULL. */
DM_API int dm_default_params(dm_params* p);

/* Create a context for H x W images and L labels (2 <= L <= 256,
 * 1 <= H, W <= 65535, H*W*L < 2^31).  Copies *p.  On success *out owns host
 * memory only; release it with dm_destroy.  DM_ERR_ARG for invalid sizes or
 * parameters.  If omega*r is not an integer table reaching its cap within 4
 * labels for w_hi or w_lo, the context is still created (the continuous
 * stage works) but dm_discrete and dm_discrete_pass return DM_ERR_ARG. */
DM_API int dm_create(int H, int W, int L, const dm_params* p, dm_ctx** out);

/* Release a context (NULL is a no-op).  Does not free the workspace. */
DM_API int dm_destroy(dm_ctx* ctx);

/* Bytes of device workspace the context needs (256-byte aligned start). */
DM_API int dm_workspace_bytes(const dm_ctx* ctx, size_t* bytes);

/* Bind caller-owned device memory of at least dm_workspace_bytes() bytes,
 * 256-byte aligned (DM_ERR_WORKSPACE otherwise).  Resets all state. */
DM_API int dm_bind_workspace(dm_ctx* ctx, void* d_workspace, size_t bytes);

/* Stream for all later work (a cudaStream_t passed as void*; NULL = 0). */
DM_API int dm_set_stream(dm_ctx* ctx, void* stream);

/* Census transform of both images and the cost volume (Sec. 3.1):
 * c[y][x][l] = popcount(census_L(y,x) ^ census_R(y,x-l)), or win*win-1 when
 * x-l < 0; census bits are [I(neighbour) < I(centre)] over the window with
 * clamp-to-edge borders.  Also computes the edge weights from d_left.
 * Resets the dual variables. */
DM_API int dm_cost_volume(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right);

/* Use a caller-made cost volume and edge weights (copied into the
 * workspace).  Resets the dual variables. */
DM_API int dm_set_cost_volume(dm_ctx* ctx, const uint8_t* d_cost, const uint8_t* d_wh,
                              const uint8_t* d_wv);

/* Use a caller-made uint16 cost volume (contexts created with
 * params.cost_bytes = 2; DM_ERR_STATE otherwise) and edge weights, copied into
 * the workspace.  cost_max bounds the samples (0..65535); the caller
 * guarantees it.  It selects the Dual MM kernel: the packed 16-bit kernel when
 * cost_max + 2 (omega C + 1) <= 16257, else the int32 kernel, which needs
 * (cost_max + 4 omega C) (max(H, W) + 1) < 2^30 (DM_ERR_RANGE otherwise).
 * Resets the dual variables. */
DM_API int dm_set_cost_volume_u16(dm_ctx* ctx, const uint16_t* d_cost, const uint8_t* d_wh,
                                  const uint8_t* d_wv, int cost_max);

/* dm_cost_volume for the next frame of a sequence, keeping the vertical duals
 * lambda_v of the previous frame as the starting point of Alg. Dual_MM (a warm
 * start; the paper starts from zero).  The first horizontal pass then uses the
 * unaries c_new + lambda_v_old; the lower bound returned after a full
 * iteration is valid for the new frame whatever lambda_v_old was, because each
 * pass rebuilds its dual from a minorant of the current chains.  Without a
 * previous cost volume this is dm_cost_volume.  A warm start whose unaries do
 * not fit the 16-bit kernel's storage is reported as DM_ERR_DEVICE by the
 * next synchronising call. */
DM_API int dm_cost_volume_warm(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right);

/* Zero both dual variables (a cold start of Alg. Dual_MM). */
DM_API int dm_reset_duals(dm_ctx* ctx);

/* One half-iteration of Alg. Dual_MM (which = 0: horizontal chains with
 * unaries c + lambda_v, writes lambda_h; which = 1: vertical chains with
 * unaries lambda_h, writes lambda_v).  For tests and instrumentation. */
DM_API int dm_discrete_pass(dm_ctx* ctx, int which);

/* iters full iterations of Alg. Dual_MM (horizontal then vertical pass)
 * from the current duals, then the labelling x_i = argmin_l
 * (lambda_h + lambda_v)_i(l) (ties: smallest l) and the lower bound
 * sum_i min_l (lambda_h + lambda_v)_i(l) of every iteration.  h_lb
 * (nullable) receives the iters bounds and makes the call synchronous. */
DM_API int dm_discrete(dm_ctx* ctx, int iters, int64_t* h_lb);

/* Primal-dual refinement (Sec. 2.4 and 3.1): iters iterations split evenly
 * over params.warps re-linearisations, starting from d_u0 (H x W float32,
 * device; NULL = the labels of the last dm_discrete).  p and q start at 0. */
DM_API int dm_refine(dm_ctx* ctx, int iters, const float* d_u0);

/* The whole path: cost volume, dmm_iters iterations of Dual MM, pd_iters
 * primal-dual iterations; the refined disparity (H x W float32) is written
 * to d_u (device). */
DM_API int dm_solve(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int dmm_iters,
                    int pd_iters, float* d_u);

/* Record dm_solve(ctx, d_left, d_right, dmm_iters, pd_iters, d_u) as a CUDA
 * graph of the context's stream (which must be a stream created by the
 * caller: the legacy stream cannot be captured, DM_ERR_STATE).  Nothing runs
 * during the capture.  dm_replay launches the graph on the context's stream:
 * each replay reads the images currently in d_left, d_right and writes d_u,
 * so the buffers must stay allocated and in place.  A new capture replaces
 * the previous one; dm_destroy releases it.  The context's state (labels,
 * duals, disparity) after a replay is that of the solve. */
DM_API int dm_capture(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right, int dmm_iters,
                      int pd_iters, float* d_u);
DM_API int dm_replay(dm_ctx* ctx);

/* dm_solve for the next frame of a sequence: dm_cost_volume_warm, then the
 * same iterations (the refinement starts from the new labels). */
DM_API int dm_solve_next(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right,
                         int dmm_iters, int pd_iters, float* d_u);

/* ---- Two-sided consistency check (Sec. 4.1.1; Table 1's caption: the full
 * left-right procedure takes twice the one-view time) ---------------------
 *
 * The right view's problem (the right image as reference, label l matching
 * the left image's pixel x + l) is the left-reference problem of the mirrored
 * pair: the right image with its columns reversed as reference, the left image
 * with its columns reversed as the other view.  Its census cost volume is the
 * right-view cost volume with columns reversed (the census bits of a mirrored
 * window are a fixed permutation of the original ones, the same on both
 * sides), so the unchanged kernels solve it. */

/* dm_cost_volume of the mirrored pair built from (d_left, d_right), both
 * H x W uint8 row-major on the device: the context then holds the right view's
 * problem in mirrored columns, and its disparity u'[y][x'] is the right view's
 * disparity at column W-1-x'.  Resets the duals. */
DM_API int dm_cost_volume_mirrored(dm_ctx* ctx, const uint8_t* d_left, const uint8_t* d_right);

/* The check itself, on caller buffers (device, H x W row-major):
 * d_u_left: the left view's disparity (float32); d_u_mirrored: the mirrored
 * problem's disparity.  The left pixel (y, x) with d = u_left[y][x] has its
 * counterpart at xr = x - rint(d) (nearest, ties to even) and passes when
 * 0 <= xr < W and |d - u_right[y][xr]| <= max_diff in single precision.
 * Writes d_ok (uint8: 1 pass, 0 fail), d_u_out (float32: d, or -1 where the
 * check fails) and, if not NULL, d_u_right (float32: the right view's
 * disparity in its own columns).  Asynchronous on stream (NULL: the legacy
 * default stream).  DM_ERR_ARG for a null buffer, H or W <= 0, or max_diff
 * negative or not finite. */
DM_API int dm_lr_check(const float* d_u_left, const float* d_u_mirrored, int H, int W,
                       float max_diff, uint8_t* d_ok, float* d_u_out, float* d_u_right,
                       void* stream);

/* Both views and the check: `left` solves (d_left, d_right) as dm_solve does,
 * `right` (another context of the same H, W, L and cost storage) solves the
 * mirrored pair, then dm_lr_check writes d_ok, d_u and d_u_right (nullable)
 * on the left context's stream.  When the two contexts have different streams
 * the right view runs on its own stream, concurrently with the left view: it
 * starts after the work queued on the left stream so far (the inputs), and
 * the left stream waits for it before the check.  Each context keeps its own
 * labels, duals and disparity for the getters.  DM_ERR_ARG for mismatched
 * contexts (or the same context twice) and as dm_lr_check. */
DM_API int dm_solve_lr(dm_ctx* left, dm_ctx* right, const uint8_t* d_left, const uint8_t* d_right,
                       int dmm_iters, int pd_iters, float max_diff, uint8_t* d_ok, float* d_u,
                       float* d_u_right);

/* Same with host buffers: copies the images in and the disparity (and, if
 * h_labels is not NULL, the labels) out through the workspace; synchronous. */
DM_API int dm_solve_host(dm_ctx* ctx, const uint8_t* h_left, const uint8_t* h_right,
                         int dmm_iters, int pd_iters, float* h_u, uint16_t* h_labels);

/* Copies of internal state into caller device buffers. */
DM_API int dm_get_labels(dm_ctx* ctx, uint16_t* d_labels);            /* H*W        */
DM_API int dm_get_disparity(dm_ctx* ctx, float* d_u);                 /* H*W        */
DM_API int dm_get_duals(dm_ctx* ctx, int32_t* d_lam_h, int32_t* d_lam_v); /* H*W*L each */
DM_API int dm_get_cost_volume(dm_ctx* ctx, uint8_t* d_cost, uint8_t* d_wh, uint8_t* d_wv);
                                       /* d_cost: H*W*L*cost_bytes bytes */

/* Lower bounds of the last dm_discrete call (n <= iters of that call);
 * synchronous. */
DM_API int dm_get_lower_bounds(dm_ctx* ctx, int64_t* h_lb, int n);

/* Continuous energy E(u) = sum alpha D_i(u_i) + sum lambda_r omega r((Au)_e)
 * (Eq. mrf_formulation) of the current disparity; synchronous. */
DM_API int dm_energy(dm_ctx* ctx, double* h_energy);

/* ---- Differentiable refinement -------------------------------------------
 * The refinement of dm_refine is a fixed sequence of primal-dual iterations
 * (Eq. cont_iterates) with a re-linearised data term (Sec. 3.1); these calls
 * give it on a float32 cost volume and its reverse mode: gradients of a loss
 * of the refined disparity with respect to the cost volume, the per-pixel
 * data weights alpha and the regularisation weight lambda_r.  The paper runs
 * the iteration forward only; the reverse follows the chain rule through the
 * same iterates, with every piecewise-linear prox differentiated on the branch
 * the forward took (at a tie, the branch whose slope in its argument is 0).
 */

/* Continuous stage on a caller's float32 cost volume d_cost [H][W][L]
 * (device, 4-byte aligned).  The context BORROWS d_cost: it must stay valid
 * and unchanged until the next dm_set_cost_volume*, dm_cost_volume or
 * dm_destroy.  d_wh, d_wv ([H][W] uint8 edge weights) are copied; both NULL
 * keeps the weights of an earlier dm_cost_volume / dm_set_cost_volume
 * (DM_ERR_STATE if there are none).  While a float cost volume is set the
 * discrete stage returns DM_ERR_STATE (its arithmetic is integer); dm_refine,
 * dm_energy and the calls below use the float samples.  Labels of an earlier
 * dm_discrete stay available as a starting point. */
DM_API int dm_set_cost_volume_f32(dm_ctx* ctx, const float* d_cost, const uint8_t* d_wh,
                                  const uint8_t* d_wv);

/* Per-pixel data-term weights alpha_i (d_alpha: [H][W] float32, device,
 * borrowed like d_cost above) in place of the scalar params.alpha; NULL
 * returns to the scalar.  Applies to dm_refine, dm_energy and the calls
 * below. */
DM_API int dm_set_data_weights(dm_ctx* ctx, const float* d_alpha);

/* Regularisation weight lambda_r of the continuous stage (>= 0, finite). */
DM_API int dm_set_lambda_r(dm_ctx* ctx, double lambda_r);

/* Bytes of device tape that dm_refine_tape needs for iters iterations with a
 * checkpoint every ckpt_every iterations (>= 1).  The tape holds the state
 * (u, p, q: five H x W float32 arrays) at every checkpoint and at every warp
 * start, room to recompute one segment, and the reverse pass's scratch. */
DM_API int dm_tape_bytes(const dm_ctx* ctx, int iters, int ckpt_every, size_t* bytes);

/* dm_refine with checkpoints: the same iterations and result (read with
 * dm_get_disparity), and the states needed by dm_refine_backward written to
 * d_tape (device, 256-byte aligned, >= dm_tape_bytes; DM_ERR_WORKSPACE
 * otherwise).  d_u0 as in dm_refine. */
DM_API int dm_refine_tape(dm_ctx* ctx, int iters, int ckpt_every, const float* d_u0, void* d_tape,
                          size_t tape_bytes);

/* Reverse mode of the last dm_refine_tape on this context (the same d_tape
 * and tape_bytes; DM_ERR_STATE if the tape or any input changed since).
 * d_gu: d loss / d u of the refined disparity ([H][W] float32).  Outputs,
 * each nullable and overwritten: d_gcost [H][W][L] float32 (d loss / d cost),
 * d_galpha [H][W] float32 (d loss / d alpha_i; with a scalar alpha the
 * derivative in it is the sum), d_glambda one float64 (d loss / d lambda_r),
 * d_gu0 [H][W] float32 (d loss / d u0).  Each segment between checkpoints is
 * recomputed from its checkpoint, then reversed one iteration per kernel.  The
 * tape stays valid: the call may be repeated with another d_gu. */
DM_API int dm_refine_backward(dm_ctx* ctx, const float* d_gu, void* d_tape, size_t tape_bytes,
                              float* d_gcost, float* d_galpha, double* d_glambda, float* d_gu0);

/* Forward mode of the same refinement: runs dm_refine(iters, d_u0) (result
 * readable with dm_get_disparity) and writes to d_du ([H][W] float32) the
 * directional derivative of the refined disparity in the direction
 * (d_du0, d_dcost, d_dalpha, dlambda) of (u0, the float cost volume, alpha,
 * lambda_r); NULL directions are zero.  Derivatives are taken on the branches
 * the forward takes, as in dm_refine_backward, so for any direction v and
 * any d_gu the pair satisfies <d_gu, J v> = <J^T d_gu, v>.  d_scratch:
 * device, 256-byte aligned, >= dm_jvp_bytes (15 H x W float32 arrays). */
DM_API int dm_jvp_bytes(const dm_ctx* ctx, size_t* bytes);
DM_API int dm_refine_jvp(dm_ctx* ctx, int iters, const float* d_u0, const float* d_du0,
                         const float* d_dcost, const float* d_dalpha, double dlambda, float* d_du,
                         void* d_scratch, size_t scratch_bytes);

/* ---- Batched form ---------------------------------------------------------
 * n stereo pairs of mixed sizes and label counts solved together: every pair
 * has its own context (same parameters) on a slice of one workspace, and the
 * Dual MM passes and primal-dual iterations run as persistent kernels over all
 * pairs (one launch per label class and pass, one per iteration).  The batch
 * runs on a stream of its own (dm_batch_set_stream; a non-default stream is
 * needed for capture).  Results per pair are read through dm_batch_context
 * and the single-pair getters.  The paper solves one pair at a time.
 */
typedef struct dm_batch dm_batch;

/* H, W, L: arrays of n sizes (each as in dm_create). */
DM_API int dm_batch_create(int n, const int* H, const int* W, const int* L, const dm_params* p,
                           dm_batch** out);
DM_API int dm_batch_destroy(dm_batch* b);
DM_API int dm_batch_workspace_bytes(const dm_batch* b, size_t* bytes);
DM_API int dm_batch_bind_workspace(dm_batch* b, void* d_workspace, size_t bytes);
DM_API int dm_batch_set_stream(dm_batch* b, void* stream);
/* The context of pair i (owned by the batch; do not destroy or rebind it). */
DM_API int dm_batch_context(dm_batch* b, int i, dm_ctx** out);

/* Solve every pair: cost volume, dmm_iters (1..256) Dual MM iterations,
 * pd_iters primal-dual iterations; d_left, d_right: n device image pointers
 * (host array); d_u: n device outputs (host array, entries nullable; NULL for
 * none).  Asynchronous. */
DM_API int dm_batch_solve(dm_batch* b, const uint8_t* const* d_left, const uint8_t* const* d_right,
                          int dmm_iters, int pd_iters, float* const* d_u);

/* Record one dm_batch_solve with these arguments into a CUDA graph owned by the
 * batch (nothing runs); dm_batch_replay launches it.  The graph keeps the
 * pointers: new inputs are written into the same image buffers between
 * replays.  Changing the stream, workspace or tuning drops the graph. */
DM_API int dm_batch_capture(dm_batch* b, const uint8_t* const* d_left,
                            const uint8_t* const* d_right, int dmm_iters, int pd_iters,
                            float* const* d_u);
DM_API int dm_batch_replay(dm_batch* b);

/* Synchronise the stream and report a device-side error of any pair. */
DM_API int dm_batch_sync(dm_batch* b);

/* Launch shapes: choice[5] = {CTAs per SM of the persistent Dual MM kernels
 * (1-3), primal-dual tile width, tile height (32x8, 32x4, 32x16, 64x4, 64x8,
 * 16x16), CTAs per SM of the persistent primal-dual kernel (1-64), group
 * budget in MB: consecutive pairs whose Dual MM working set (duals and costs)
 * fits it are solved together, both stages, before the next group (0: one
 * group)}.
 * dm_batch_tune times every candidate on these inputs (it runs the cost volumes
 * and one iteration of both stages first; synchronous) and keeps the fastest;
 * with cache_path (nullable) it first looks for a line for this GPU, these
 * shapes and this penalty, and appends its result.  Results do not depend on
 * the choice. */
DM_API int dm_batch_tune(dm_batch* b, const uint8_t* const* d_left, const uint8_t* const* d_right,
                         const char* cache_path, int* choice);
DM_API int dm_batch_set_tuning(dm_batch* b, const int* choice);
DM_API int dm_batch_get_tuning(const dm_batch* b, int* choice);

/* Kernels enqueued for the batch (a replay counts the graph's kernels). */
DM_API int dm_batch_launch_count(const dm_batch* b, uint64_t* count);

/* One Dual MM pass (which = 0 horizontal, 1 vertical) over every pair of a
 * batch that has been solved or captured before, with the persistent kernels
 * of the solve, on the batch's stream; for instrumentation.  It continues from
 * the current duals and adds the pass's bound to the first lower-bound slot.
 * DM_ERR_STATE before the first solve or capture. */
DM_API int dm_batch_discrete_pass(dm_batch* b, int which);

/* Allocation-free variant of dm_discrete_pass.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * (a fixed memory budget decided at start-up, a real-time or embedded
 * pipeline that forbids allocation while running, or an environment where
 * cudaMalloc is unavailable).  It needs no context and no workspace and calls
 * no allocating routine: the caller passes the inputs and the output, all
 * device pointers on the current device, and the pass's scratch lives in a
 * fixed 32 MiB device array inside libdm.so that every GPU loading the
 * library holds until the process exits.
 *   which = 0: horizontal chains, unaries d_cost + d_lam_in (d_lam_in =
 *              lambda_v), d_wedge = wh, writes d_lam_out = lambda_h;
 *   which = 1: vertical chains, unaries d_lam_in (= lambda_h), d_wedge = wv,
 *              writes d_lam_out = lambda_v (d_cost may be NULL).
 * Layouts are those of the context API ([H][W][L] uint8 cost, [H][W] uint8
 * weights, [H][W][L] int32 duals); *p supplies the penalty (checked as by
 * dm_create; the pass always uses the hierarchical minorant and reads uint8
 * costs, whatever p->cost_bytes says).  d_err (required, a caller-zeroed device
 * int32) receives nonzero bits if an edge weight has no integer penalty table;
 * d_lam_out must not be d_lam_in.  Asynchronous on `stream` (a cudaStream_t as
 * void*).  The pass runs in int32: with P2 the largest omega C over every
 * omega with a penalty table and n = max(H, W) + 1, it needs
 * (255 + Lambda + 4 P2) n < 2^30 where Lambda bounds |d_lam_in|; the call
 * returns DM_ERR_RANGE when this fails already for Lambda = 0 and relies on the
 * caller for d_lam_in (the duals that Dual MM itself produces from such costs
 * stay within it).  Limit: 2 * H * W * KP * 4 bytes <= 32 MiB - 8.25 KiB, where
 * KP is L rounded up to 32, 64, 128 or 256; larger problems return
 * DM_ERR_WORKSPACE before any work is enqueued.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first
 * call before any stream capture.  All calls share the one array: calls whose
 * work overlaps on the GPU race. */
DM_API int dm_discrete_pass_noalloc(int H, int W, int L, const dm_params* p, int which,
                                    const uint8_t* d_cost, const uint8_t* d_wedge,
                                    const int32_t* d_lam_in, int32_t* d_lam_out,
                                    int32_t* d_err, void* stream);

/* ---- Optical flow (Sec. 2.2 "Flow"; the appendix section on optical flow) --
 *
 * Images I1, I2 (H x W uint8); the displacement of pixel (y, x) is
 * (d1, d2) = (lo1 + label1, lo2 + label2), d1 horizontal, with label_k in
 * [0, K_k).  The data cost is D(d1, d2) = popcount(census1(y, x) ^ census2(y + d2,
 * x + d1)), win*win - 1 where the displaced pixel leaves the image.  The two
 * components are two layers, each an ordinary context: layer1 with L = K1,
 * layer2 with L = K2, the same H, W and census window, uint8 cost storage.
 *
 * The discrete stage is decoupled (Eq. flow decoupled costs): layer k gets the
 * cost min over the other component of D, and the edge weights of I1; each
 * layer then runs dm_discrete as a stereo problem (the two may run
 * concurrently on different streams).
 *
 * The continuous stage refines both components together with the quadratic
 * model of the data term at the start of each of params.warps warps: central
 * finite differences with step h for the gradient L and the Hessian Q of
 * alpha * D (D bilinear between the integer displacements, arguments clamped
 * to the ranges), Q replaced by its positive-semidefinite part; the prox is
 * u = (I + tau Q)^-1 (u^ + tau (Q u0 - L)), each component then clamped to
 * [u0 - h, u0 + h] within its range.  The regulariser is lambda_r omega r of
 * each component separately.  The iterates are those of dm_refine. */

/* Census of both images, edge weights of I1 and the two decoupled cost
 * volumes (written into layer1 and layer2), on layer1's stream; layer2's
 * stream waits for it.  Resets both layers' duals.  DM_ERR_ARG for
 * mismatched layers or |lo| > 65535, DM_ERR_STATE without a workspace or with
 * uint16 cost storage. */
DM_API int dm_flow_cost_volumes(dm_ctx* layer1, dm_ctx* layer2, const uint8_t* d_img1,
                                const uint8_t* d_img2, int lo1, int lo2);

/* Bytes of caller scratch (device, 256-byte aligned) dm_flow_refine needs. */
DM_API int dm_flow_refine_bytes(int H, int W, size_t* bytes);

/* iters primal-dual iterations of the flow from the labels of the last
 * dm_discrete of each layer (after dm_flow_cost_volumes on the same layers),
 * on layer1's stream after the work queued on layer2's.  Writes the
 * displacements d_u1 = lo1 + u1, d_u2 = lo2 + u2 (H x W float32, device).
 * DM_ERR_STATE without the cost volumes or the labels, DM_ERR_WORKSPACE for a
 * small or misaligned scratch. */
DM_API int dm_flow_refine(dm_ctx* layer1, dm_ctx* layer2, int iters, void* d_scratch,
                          size_t bytes, float* d_u1, float* d_u2);

/* ---- Chain minorant of the Dual MM passes (Sec. 2.3 "Good and Fast
 * Minorants"; App. A) ------------------------------------------------------
 *
 * DM_MINORANT_HIER (the default): the hierarchical minorant of Alg. Handshake.
 * DM_MINORANT_NAIVE: every node of a chain takes its min-marginal m_i divided
 *   by the chain length n, rounded down: floor(m_i / n).
 * DM_MINORANT_ITERATIVE (Alg. iterative-minorant): mu := 0, then max_pass
 *   passes over the chain, forward first and then alternating; at each node the
 *   min-marginal m_i of the remainder f - mu is drained by mu_i +=
 *   floor(gamma m_i), gamma = gamma_num / gamma_den on every pass but the last,
 *   where gamma = 1 (the minorant is then maximal).
 * Both alternatives run on the int32 kernel (one warp per chain) and give the
 * same numbers as the oracle.  Changing the minorant of a context that holds a
 * cost volume chooses the dual storage again and resets the duals.
 * DM_ERR_ARG for an unknown kind or, for the iterative minorant, max_pass
 * outside [1, 64], gamma_den outside [1, 1024] or gamma_num outside
 * [0, gamma_den]; the other arguments are ignored for the first two kinds.
 * The batched form uses the hierarchical minorant only (a batch whose context
 * was switched reports DM_ERR_STATE). */
#define DM_MINORANT_HIER      0
#define DM_MINORANT_NAIVE     1
#define DM_MINORANT_ITERATIVE 2
DM_API int dm_set_minorant(dm_ctx* ctx, int kind, int max_pass, int gamma_num, int gamma_den);

/* The Dual MM kernel chosen for the current cost volume: *kernel = 8 (packed
 * 16-bit arithmetic on lane groups, 8-bit messages), 16 (packed 16-bit
 * arithmetic, one warp per chain) -- both with dual deltas of *delta_bytes
 * bytes per label -- or 32 (int32 kernel, *delta_bytes = 4).  Host only. */
DM_API int dm_get_path(const dm_ctx* ctx, int* kernel, int* delta_bytes);

/* Number of kernels this context has enqueued since dm_create (host-side
 * counter; instrumentation for benchmarks). */
DM_API int dm_launch_count(const dm_ctx* ctx, uint64_t* count);

/* Synchronise the stream and report a device-side error, if any. */
DM_API int dm_sync(dm_ctx* ctx);

/* Static description of a status code. */
DM_API const char* dm_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* DM_H */
