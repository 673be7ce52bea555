/*
 * nsm.h -- C ABI of the GB300 (sm_103a) Neural Shadow Mapping hot path.
 *
 * The library computes per-pixel shadow visibility for one view from the
 * rasterised inputs the paper names (Sec. 3.1): a G-buffer (world position,
 * view depth d, normal n), a vanilla single-frustum shadow map holding the
 * emitter-to-occluder depth z, and the emitter description (position, size).
 * Two stages run on the GPU:
 *   1. the shadow-map feature gather: project each pixel into the map, fetch
 *      z, do the depth test and form the four network inputs
 *      f = [c_e + r_e, z / z_f, z - z_f, c_c / d]   (Sec. 3.1, 3.2, Fig. 2);
 *   2. the compact encoder/decoder (Sec. 3.5): 3 levels of widths 16/32/64,
 *      one 3x3 and one 1x1 convolution per level, 2x2 average pooling down,
 *      bilinear x2 upsampling up, decoder skip merged by a sum, no skip at
 *      level 0, ReLU after every convolution, 1x1 head 16 -> 1 + sigmoid.
 *
 * Conventions for every entry point:
 *   - Buffers named "device" must be device (or managed) memory of the
 *     current CUDA device, owned by the caller; the library never frees them.
 *   - Images are dense, row-major, row 0 first; pixel p = y * W + x.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) and never synchronise, except
 *     where stated.  Errors found on the host are returned before any work is
 *     queued; outputs are then untouched.  nsm_last_error() gives a message.
 *   - No entry point allocates device memory except nsm_ctx_create,
 *     nsm_weights_create and nsm_train_state_create (set-up calls).
 *   - Kernel waits are bounded; a wait that runs out sets the context's device
 *     error word, read back by nsm_ctx_check (NSM_ERR_TIMEOUT).
 */
#ifndef NSM_H
#define NSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NSM_ABI_VERSION 1

typedef enum {
    NSM_OK = 0,
    NSM_ERR_INVALID_ARG = 1,  /* null / non-device pointer, bad enum, bad value */
    NSM_ERR_SHAPE = 2,        /* unsupported sizes (see each call) */
    NSM_ERR_ALIGNMENT = 3,    /* a pointer or size breaks the stated alignment */
    NSM_ERR_DEVICE = 4,       /* no usable sm_103 device / wrong device */
    NSM_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    NSM_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    NSM_ERR_UNSUPPORTED = 7,  /* valid request this build cannot serve */
    NSM_ERR_WORKSPACE = 8     /* workspace missing or too small */
} nsm_status;

typedef enum {
    NSM_FP32 = 0,  /* FP32 CUDA-core convolutions (parity form) */
    NSM_BF16 = 1,  /* BF16 operands on tcgen05 tensor cores, FP32 accumulation */
    NSM_FP8 = 2    /* FP8 E4M3 operands (per-channel weight scales), FP32 accumulation */
} nsm_precision;

/* Emitter and its shadow-map frustum (Sec. 3.1). */
typedef struct {
    float pos[3];         /* emitter centre L, world space */
    float radius;         /* emitter radius r (world); 0 = point light */
    float r_hat;          /* emitter-size input, added to c_e as a DC offset (Sec. 3.1.1), 0..4 */
    float view_proj[16];  /* world -> light clip space, row-major:
                             clip_r = ((M[r][0] Px + M[r][1] Py) + M[r][2] Pz) + M[r][3] */
    float z_far;          /* depth used for pixels that project outside the map */
    float bias;           /* relative depth bias beta: a pixel is lit iff z_f <= z + beta z_f */
    float tan_half_fov;   /* tan(fov / 2) of the map frustum (blocker-search window) */
} nsm_light;

typedef struct {
    float pos[3];         /* camera centre C, world space */
} nsm_camera;

/* One view: G-buffer + shadow map + emitter + camera. */
typedef struct {
    int H, W;             /* view size in pixels */
    const float* pos4;    /* device, H*W*4 floats, 16-byte aligned: (P.x, P.y, P.z, d), d > 0 the view depth */
    const float* nrm4;    /* device, H*W*4 floats, 16-byte aligned: (n.x, n.y, n.z, unused), |n| = 1 */
    int Hs, Ws;           /* shadow-map size (texels), each in [1, 16384] */
    const float* sm;      /* device, Hs*Ws floats: z per texel, row j = floor(v Hs), v = ndc_y / 2 + 1/2 */
    nsm_light light;
    nsm_camera camera;
} nsm_frame;

typedef struct nsm_ctx nsm_ctx;          /* device error word, autotune table, graph cache */
typedef struct nsm_weights nsm_weights;  /* network weights, FP32 + packed BF16 / FP8 copies */

/* ---------------------------------------------------------------- general */

int nsm_abi_version(void);

/* Message for the last error returned on the calling thread ("" if none). */
const char* nsm_last_error(void);

/* Create a context on the current CUDA device (which must be sm_103). Allocates
 * a few bytes of device memory (the error word). */
nsm_status nsm_ctx_create(nsm_ctx** out);
void nsm_ctx_destroy(nsm_ctx* ctx);

/* Synchronise the context's work and read the device error word: NSM_OK, or
 * NSM_ERR_TIMEOUT when a bounded device wait gave up since the last check
 * (the word is cleared).  This call synchronises the device. */
nsm_status nsm_ctx_check(nsm_ctx* ctx);

/* Profiling hook.  With n > 0, every later nsm_infer / nsm_infer_host on this
 * context records events[i] (cudaEvent_t handles passed as void*, created and
 * owned by the caller) on its stream right before launching its i-th kernel,
 * and events[k] after the last of its k kernels; n must be >= k + 1 for the
 * precision used (see nsm_infer_kernel_count).  n = 0 (events NULL) turns the
 * hook off.  Recording events does not change the results. */
nsm_status nsm_ctx_set_stage_events(nsm_ctx* ctx, void* const* events, int n);

/* Number of kernels nsm_infer launches per call for a precision, and the name
 * of the i-th (a static string; "" when i is out of range). */
int nsm_infer_kernel_count(nsm_precision precision);
const char* nsm_infer_kernel_name(nsm_precision precision, int i);

/* ---------------------------------------------------------------- weights */

/* Number of floats in the canonical parameter vector: for each layer, in the
 * order enc0_3x3, enc0_1x1, enc1_3x3, enc1_1x1, bott_3x3, bott_1x1, dec1_3x3,
 * dec1_1x1, dec0_3x3, dec0_1x1, head, its OIHW weights then its bias
 * (39,248 weights + 273 biases = 39,521; Sec. 3.5, suppl. Table 5). */
size_t nsm_param_count(void);

/* Upload a canonical parameter vector (host memory, n == nsm_param_count())
 * and build the packed BF16 / FP8 copies.  Set-up call: allocates device memory. */
nsm_status nsm_weights_create(nsm_ctx* ctx, const float* host_params, size_t n, nsm_weights** out);

/* Network topologies.  NSM_TOPO_LEVELS3: the 3-level encoder/decoder above.
 * NSM_TOPO_S2D: the paper's first-layer optimisation (Sec. 3.5): the level-0
 * convolutions removed, each 2x2 square of pixels flattened into 16 input
 * channels (channel 4 (2a + b) + c = feature c of square offset (a, b)) that
 * feed the level-1 encoder, and a 1x1 head 16 -> 4 whose channel 0 is upscaled
 * bilinearly to full resolution and whose channels 1, 2, 3 are added at square
 * offsets (0, 1), (1, 0), (1, 1) before the sigmoid.  Parameter order:
 * enc1_3x3, enc1_1x1, bott_3x3, bott_1x1, dec1_3x3, dec1_1x1, head (16 -> 4),
 * each OIHW weights then bias (35,904 weights + 212 biases = 36,116). */
typedef enum { NSM_TOPO_LEVELS3 = 0, NSM_TOPO_S2D = 1 } nsm_topology;
size_t nsm_param_count_topology(nsm_topology topology);  /* 0 for an unknown topology */
/* nsm_weights_create for a topology (nsm_weights_create = NSM_TOPO_LEVELS3).
 * Weights of NSM_TOPO_S2D run in nsm_infer / nsm_infer_host with NSM_BF16
 * only (other precisions, the batched calls, the autotuner and training
 * return NSM_ERR_UNSUPPORTED for them). */
nsm_status nsm_weights_create_topology(nsm_ctx* ctx, nsm_topology topology, const float* host_params, size_t n,
                                       nsm_weights** out);

/* Re-pack from a canonical FP32 vector already on the device (e.g. the
 * master weights of a training state); asynchronous on stream. */
nsm_status nsm_weights_load_device(nsm_weights* w, const float* dev_params, size_t n, void* stream);
void nsm_weights_destroy(nsm_weights* w);

/* ---------------------------------------------------------------- gather */

/* Feature gather (Sec. 3.1, 3.2): for every pixel p of the frame
 *   feat_out  [4][H][W] float32 (device, required):
 *             channel 0 c_e + r_hat, 1 z / z_f, 2 z - z_f, 3 c_c / d, with
 *             z_f = |L - P|, c_e = n.(L - P) / z_f, c_c = n.(C - P) / |C - P|;
 *   texel_out [H][W] int32 (device, nullable): j * Ws + i of the texel read,
 *             -1 when P projects outside the map (then z = z_far);
 *   hard_out  [ceil(H W / 32)] uint32 (device, nullable): bit (p % 32) of
 *             word p / 32 is 1 iff the pixel is lit by the hard depth test;
 *   blocker_out [3][H][W] float32 (device, nullable): z_min, z_max of the map
 *             texels z < z_f - beta z_f within the emitter's window around
 *             (i, j) (half-size k = min(32, ceil(r Ws / 2 / (z_f tan_half_fov)))),
 *             and the penumbra width x_a + x_b of the spherical-occluder model
 *             (Sec. 3.6, suppl. Sec. 4); all three 0 where no blocker is found.
 * Texel index, hard bit and blocker window are computed in binary32 with a
 * fixed operation order and no contraction, so they are reproducible bit for
 * bit.  H, W >= 0 (0 = nothing to do).  With blocker_out the call takes
 * Ws * Hs * 16 bytes of device scratch (the map's 8 x 8 and 4 x 4 min / max
 * tables) from a library-owned pool, in stream order, for the duration of its
 * kernels; NSM_ERR_CUDA if that allocation fails.  nsm_features_ws takes that
 * scratch from the caller instead (no allocation): workspace (device, 256-byte
 * aligned) of nsm_features_workspace_bytes(Hs, Ws) bytes when blocker_out is
 * given, NSM_ERR_WORKSPACE if missing or short; ignored otherwise. */
nsm_status nsm_features(const nsm_frame* frame, float* feat_out, int32_t* texel_out,
                        uint32_t* hard_out, float* blocker_out, void* stream);
size_t nsm_features_workspace_bytes(int Hs, int Ws);
nsm_status nsm_features_ws(const nsm_frame* frame, float* feat_out, int32_t* texel_out, uint32_t* hard_out,
                           float* blocker_out, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- inference */

/* Bytes of device workspace nsm_infer needs for an H x W view (0 if H or W
 * is 0).  The workspace holds the intermediate activations of the levels,
 * 4 bytes per channel (FP32, or a BF16 hi + lo pair in the BF16 form). */
size_t nsm_infer_workspace_bytes(int H, int W, nsm_precision precision);

/* Per-pixel visibility in [0, 1] for one view: the gather fused into the
 * first level, then the network (Sec. 3.5).  Forms:
 *   NSM_FP32  CUDA cores, FP32 throughout.
 *   NSM_BF16  tcgen05 tensor cores, every operand a BF16 hi + lo pair (weights,
 *             features, activations), FP32 accumulation: ~2^-16 relative
 *             storage error.
 *   NSM_FP8   tcgen05 tensor cores, E4M3 operands: weights with one scale per
 *             output channel, activations and features with unit scale
 *             (saturating at +-448), FP32 accumulation.
 * The texel index and the depth test are FP32 (bit-exact) in every form.
 *   vis_out   [H][W] float32 (device).
 *   workspace device, >= nsm_infer_workspace_bytes(H, W, precision) bytes,
 *             256-byte aligned, not shared with a concurrent call.
 * H and W must be multiples of 4 (two 2x2 poolings), W <= 16384, H <= 16384. */
nsm_status nsm_infer(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w,
                     nsm_precision precision, void* workspace, size_t workspace_bytes,
                     float* vis_out, void* stream);

/* nsm_infer with HOST inputs and output: copies pos4 / nrm4 / sm (host
 * pointers inside *frame, pinned or pageable) to the caller's device staging
 * buffers, runs nsm_infer and copies the visibility back to vis_host.
 *   dev_stage  device, >= nsm_infer_host_stage_bytes(frame) bytes, 256-byte aligned.
 * Synchronises the stream before returning (vis_host is then valid). */
size_t nsm_infer_host_stage_bytes(int H, int W, int Hs, int Ws);
nsm_status nsm_infer_host(nsm_ctx* ctx, const nsm_frame* host_frame, const nsm_weights* w,
                          nsm_precision precision, void* dev_stage, size_t stage_bytes,
                          void* workspace, size_t workspace_bytes, float* vis_host, void* stream);

/* nsm_infer_host over a sequence of n frames (frames[i]: host pointers, pinned
 * for the copies to overlap; sizes may differ), pipelined: while frame i runs
 * on `stream`, frame i + 1's G-buffer and map are copied to the device and
 * frame i - 1's visibility is copied to vis_host[i - 1] (two copy streams
 * owned by the context, events between them).  dev_stage holds 2 or 3
 * staging slots of nsm_infer_host_stage_bytes of the largest frame (rounded
 * up to 256 bytes) each: stage_bytes / slot slots are used (at most 3; fewer
 * than 2 is NSM_ERR_WORKSPACE); a slot is refilled only after the read-back
 * of the frame that used it.  workspace as for nsm_infer (largest frame).
 * Every frame's results equal nsm_infer's on the same inputs.  Synchronises
 * before returning (all vis_host[i] are then valid); on an error the copies
 * already issued are waited for. */
nsm_status nsm_infer_host_sequence(nsm_ctx* ctx, int n, const nsm_frame* frames, const nsm_weights* w,
                                   nsm_precision precision, void* dev_stage, size_t stage_bytes,
                                   void* workspace, size_t workspace_bytes, float* const* vis_host,
                                   void* stream);

/* Rows [y0, y1) of a frame's visibility, computed from the slab of rows
 * [y0 - halo, y1 + halo) clipped to the frame: the unit of a single frame
 * split across GPUs (each device takes a band of rows and recomputes its halo
 * locally; no exchange).  The network's receptive field reaches fewer than 16
 * rows, so with halo >= 16 the rows equal those of nsm_infer on the whole frame
 * bit for bit in every form (the stage kernels' per-pixel arithmetic does not
 * depend on where a tile starts); smaller halos give an approximation near the
 * band edges.  y0, y1, halo multiples of 4 (the pooling grid), 0 <= y0 < y1 <= H;
 * otherwise NSM_ERR_SHAPE.  frame as for nsm_infer (the whole frame's buffers);
 * vis_rows device, (y1 - y0) * W floats; workspace >=
 * nsm_infer_rows_workspace_bytes(...), 256-byte aligned.  Asynchronous on stream. */
size_t nsm_infer_rows_workspace_bytes(int H, int W, int y0, int y1, int halo, nsm_precision precision);
nsm_status nsm_infer_rows(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w, nsm_precision precision, int y0,
                          int y1, int halo, void* workspace, size_t workspace_bytes, float* vis_rows, void* stream);

/* ---------------------------------------------------------------- batched serving */

/* One view of a batch: its inputs (as for nsm_infer) and its output. */
typedef struct {
    nsm_frame frame;   /* H, W multiples of 4; device buffers */
    float* vis_out;    /* device [H][W] visibility */
} nsm_view;

/* Workspace bytes of nsm_infer_batched / nsm_autotune for these views (0 if invalid). */
size_t nsm_infer_batched_workspace_bytes(int n, const nsm_view* views);

/* BF16 tensor-core inference of n (1..32) independent views of any sizes
 * (different resolutions, shadow maps, emitters and cameras) in one pass of
 * five persistent kernel launches, one per network stage, whose CTAs share
 * one list of tiles of all views.  With nsm_ctx_set_graph(ctx, 1) the five
 * launches are captured once into a CUDA graph per batch plan (the views'
 * sizes and the tile plan) and replayed by a single graph launch while the
 * plan repeats (new buffers and emitters only update the graph's kernel
 * arguments).  The tile heights and CTAs per SM of every stage come from the
 * context's plan (nsm_autotune).  workspace: device, 256-byte aligned,
 * >= nsm_infer_batched_workspace_bytes.  Asynchronous on stream. */
nsm_status nsm_infer_batched(nsm_ctx* ctx, int n, const nsm_view* views, const nsm_weights* w, void* workspace,
                             size_t workspace_bytes, void* stream);
nsm_status nsm_ctx_set_graph(nsm_ctx* ctx, int enable);
/* Graph launches of the currently cached plan since it was captured. */
int nsm_ctx_graph_replays(nsm_ctx* ctx);

/* Per-view latency of nsm_infer_batched (a serving measurement beside the
 * paper's per-frame timings, Sec. 4): with dev_records set (device, 65
 * uint64, 8-byte aligned), every later batched call writes there the
 * %globaltimer time (ns) at which its first kernel started ([0]) and the time
 * the last output pixel of view v was written ([1 + v], v < n); words
 * [33 .. 64] are the kernels' completion counters.  Read them after the call
 * has finished (e.g. after a stream synchronisation); view v's latency is
 * [1 + v] - [0].  NULL turns the records off (the default).  Costs one atomic
 * per epilogue warp and tile of the last stage. */
nsm_status nsm_ctx_set_view_timing(nsm_ctx* ctx, unsigned long long* dev_records);

/* Autotuner: time every tile height and every CTAs-per-SM choice of each of
 * the five tensor-core stages on this batch (reps timed launches each, after
 * one warm-up) and keep the fastest per stage in the context's plan, used by
 * nsm_infer (BF16) and nsm_infer_batched from then on.  Synchronises. */
nsm_status nsm_autotune(nsm_ctx* ctx, int n, const nsm_view* views, const nsm_weights* w, void* workspace,
                        size_t workspace_bytes, int reps, void* stream);
/* The plan per stage (5 entries each, nullable): tile rows, CTAs per SM
 * (0 = as many as fit), and the tuned time in ms (0 before tuning). */
nsm_status nsm_autotune_report(nsm_ctx* ctx, int* rows_out, int* ctas_out, float* ms_out);
/* The warp roles of the plan per stage (5 entries each, nullable): epilogue
 * warps (4 or 8: TMEM readers) and producer warps (input staging). */
nsm_status nsm_autotune_report_warps(nsm_ctx* ctx, int* epilogue_warps_out, int* producer_warps_out);

/* The MMA schedule of the plan per stage (5 entries): 0 = each tile's 1x1
 * convolution is issued right after its 3x3; 1 = the next tile's 3x3 is
 * issued before the previous tile's 1x1, so the tensor core works on it while
 * the epilogue turns the previous 3x3 result into the 1x1 operand. */
nsm_status nsm_autotune_report_order(nsm_ctx* ctx, int* mma_order_out);

/* Manual plan: the number of tile variants of a tensor-core stage (0 enc0,
 * 1 enc1, 2 bottleneck, 3 dec1, 4 dec0; 0 for another index), and setting a
 * stage's variant and CTAs per SM (0 = as many as fit) on the context, as
 * nsm_autotune would.  Every variant computes the same result. */
int nsm_plan_variants(int stage);
nsm_status nsm_plan_set(nsm_ctx* ctx, int stage, int variant, int ctas_per_sm);

/* ---------------------------------------------------------------- backward / training */

/* Bytes of device workspace nsm_backward needs for an H x W view. */
size_t nsm_backward_workspace_bytes(int H, int W);

/* Adjoint of the FP32 inference (the hand-written backward of the gather +
 * network, Sec. 3.5): for the visibility cotangent grad_vis ([H][W] float32,
 * device) it ADDS dL/dtheta to grad_params (device, nsm_param_count floats,
 * canonical layout) and, when grad_feat is non-NULL, writes dL/dfeatures
 * ([H][W][4] float32, pixel-major, device).  vis_out (nullable, [H][W]) receives
 * the forward visibility computed on the way.  The forward keeps only the
 * level checkpoints; each level's internals are recomputed during the backward.
 * No gradient flows to the G-buffer or shadow map (the nearest-texel lookup is
 * piecewise constant).  dev_params: device FP32 canonical vector.
 * H and W multiples of 4.  Asynchronous on stream. */
nsm_status nsm_backward(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, const float* grad_vis,
                        float* grad_params, float* grad_feat, float* vis_out, void* workspace,
                        size_t workspace_bytes, void* stream);

/* nsm_backward with the form of its contractions chosen (the 3x3 level
 * recomputations, the data gradients through them and every weight
 * gradient): NSM_FP32 (exactly nsm_backward) or NSM_BF16 (tcgen05, compensated
 * BF16 operands and FP32 accumulation, weight gradients reduced in a fixed
 * order, as nsm_train_state_set_backward_precision; the weight images and the
 * partial sums use the same workspace).  Other precisions:
 * NSM_ERR_UNSUPPORTED.  A bounded device wait that gives up sets the context's
 * error word (nsm_ctx_check). */
nsm_status nsm_backward_ex(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, const float* grad_vis,
                           float* grad_params, float* grad_feat, float* vis_out, nsm_precision precision,
                           void* workspace, size_t workspace_bytes, void* stream);

/* One training batch of the temporal-window loss (Sec. 3.3, Eq. 2). */
typedef struct {
    int B, T;                   /* items; window instances per item (T >= 1), instance 0 carries
                                   the target and the gradient, instances 1..T-1 are the perturbed
                                   inputs whose outputs enter the loss detached */
    int H, W;                   /* crop size, multiples of 4 */
    int Hs, Ws;                 /* shadow-map size (all instances) */
    const float* pos4;          /* device [T][B][H][W][4], as nsm_frame.pos4 */
    const float* nrm4;          /* device [T][B][H][W][4] */
    const float* sm;            /* device [T][B][Hs][Ws] */
    const nsm_light* lights;    /* host [T][B] */
    const nsm_camera* cameras;  /* host [T][B] */
    const float* target;        /* device [B][H][W], ray-traced visibility of instance 0 */
} nsm_batch;

typedef struct {
    float lr;       /* Adam step size */
    float alpha;    /* weight of the L1 term of L(y, y~), Eq. 2 (0.9 in the paper) */
    float beta1, beta2, eps;  /* Adam moments (0.9, 0.999, 1e-8) */
} nsm_train_cfg;

typedef struct nsm_train_state nsm_train_state;  /* FP32 master weights, Adam moments, workspace */

/* Set-up call (allocates): the master weights start from host_params
 * (nsm_param_count floats); batches up to max_B x max_T instances of H x W. */
nsm_status nsm_train_state_create(nsm_ctx* ctx, const float* host_params, size_t n, int max_B, int max_T, int H,
                                  int W, nsm_train_state** out);
void nsm_train_state_destroy(nsm_train_state* st);

/* One step: features of all B*T instances, forward with level checkpoints,
 * loss L = alpha mean|x0 - x~| + sum_i alpha mean|x0 - x_i| (per item, averaged
 * over items; the VGG-19 term of Eq. 2 is not evaluated), backward through x0
 * with recomputation, Adam update of the master weights.  loss_out (device,
 * nullable) receives the batch loss.  Asynchronous on stream. */
nsm_status nsm_train_step(nsm_ctx* ctx, nsm_train_state* st, const nsm_batch* batch, const nsm_train_cfg* cfg,
                          float* loss_out, void* stream);

/* nsm_train_step in two halves, for data parallelism (the gradient is
 * exchanged between them): nsm_train_grad computes the loss and the gradient
 * of the batch (the mean over its items) into the state without touching the
 * weights; nsm_train_apply takes one Adam step with the state's gradient.
 * nsm_train_step = nsm_train_grad + nsm_train_apply.  Asynchronous on stream. */
nsm_status nsm_train_grad(nsm_ctx* ctx, nsm_train_state* st, const nsm_batch* batch, const nsm_train_cfg* cfg,
                          float* loss_out, void* stream);
nsm_status nsm_train_apply(nsm_ctx* ctx, nsm_train_state* st, const nsm_train_cfg* cfg, void* stream);

/* Copy a state vector (n = nsm_param_count floats) to device memory dev_out,
 * or set it from device memory dev_in: what = 0 master weights, 1 gradient of
 * the last step, 2 Adam first moment, 3 Adam second moment.  Asynchronous on
 * stream. */
nsm_status nsm_train_state_read(nsm_train_state* st, int what, float* dev_out, size_t n, void* stream);
nsm_status nsm_train_state_write(nsm_train_state* st, int what, const float* dev_in, size_t n, void* stream);

/* Form of the forward passes of the detached instances x_1 .. x_{T-1} of
 * Eq. 2 (Sec. 3.3: their outputs enter the loss with the gradient stopped, so
 * they are pure inference): NSM_FP32 (default; the FP32 training kernels) or
 * NSM_BF16 (the compensated-BF16 tcgen05 stage kernels of nsm_infer, up to 32
 * instances per launch, with BF16 images of the master weights packed on the
 * device at every step).  x_0 and the whole backward stay FP32.  Other
 * precisions: NSM_ERR_UNSUPPORTED. */
nsm_status nsm_train_state_set_detached_precision(nsm_train_state* st, nsm_precision precision);

/* Form of the forward pass of the target instances x_0, whose level outputs
 * the backward recomputes from: NSM_FP32 (default; the FP32 training kernels)
 * or NSM_BF16 (the compensated-BF16 tcgen05 stage kernels: the checkpoints
 * carry their ~2^-16 relative rounding, the ones stored as BF16 pairs are
 * converted to FP32 in place, and the backward stays FP32).  With both this
 * and the detached form in BF16, every forward pass of a step runs on the
 * tensor cores.  Other precisions: NSM_ERR_UNSUPPORTED. */
nsm_status nsm_train_state_set_forward_precision(nsm_train_state* st, nsm_precision precision);

/* Form of the backward's contractions (Sec. 3.3, Eq. 2 adjoint): the
 * recomputed 3x3 pre-activations of every level, the data gradients through
 * them (the transposed, flipped weights) and the weight and bias gradients of
 * every 3x3 and 1x1 layer.  NSM_FP32 (default; FP32 CUDA-core kernels, the 3x3
 * weight gradients summed with atomics, so their last bits vary from run to
 * run) or
 * NSM_BF16 (tcgen05: implicit GEMMs for the 3x3 convolutions and a GEMM over
 * the pixels for each 3x3 weight gradient, with compensated BF16 operands:
 * activations, gradients and weights as hi + lo BF16 pairs, all four products
 * accumulated in FP32 in tensor memory, ~2^-16 relative per operand; weight
 * images packed on the device at every step; the 1x1 layers' weight gradients,
 * memory-bound, in FP32 on CUDA cores; every weight gradient, the head's
 * included, reduced from per-CTA partial sums in a fixed order, so the
 * gradient is the same bits from run to run on one device).  Tensors stay
 * FP32 between the layers; the 1x1 layers' recomputations (in the 3x3
 * kernels' epilogues) and data gradients stay FP32.  A bounded device wait that gives up sets the context's error
 * word (nsm_ctx_check: NSM_ERR_TIMEOUT, code 7 or 8).  Other precisions:
 * NSM_ERR_UNSUPPORTED. */
nsm_status nsm_train_state_set_backward_precision(nsm_train_state* st, nsm_precision precision);

/* The visibility of every instance of the last nsm_train_grad / nsm_train_step
 * call on this state, [T][B][H][W] floats (n = B T H W) into device memory:
 * x_0 of every item, then the detached instances.  Asynchronous on stream. */
nsm_status nsm_train_state_read_vis(nsm_train_state* st, float* dev_out, size_t n, void* stream);

/* ---------------------------------------------------------------- scene generation (GPU ray casting) */

/* Training data as the method uses it (Sec. 3.1: a G-buffer and shadow-map
 * pass, ray-traced hard / soft shadow targets), produced on the GPU by ray
 * casting an analytic scene: the ground plane z = 0 (normal +z) plus up to 256
 * objects, each 5 floats (type, cx, cy, cz, s): type 0 = sphere of radius s,
 * type 1 = axis-aligned box of half-extent s (host array).  Nearest hit wins;
 * an exact tie goes to the lower object index and the plane is tested last.
 * FP32 arithmetic.  Asynchronous on stream; outputs on the device. */

/* cam (host, 14 floats): eye C[3], forward[3], right[3], up[3] (orthonormal),
 * tan(fovy / 2), aspect W / H.  Ray through pixel (x, y) centre, row 0 at the
 * top.  pos4 [H][W] float4 = (P, view depth (P - C).forward), nrm4 [H][W]
 * float4 = (n, 0), mask [H][W] uint8 = 1 where the ray hits (pos4 = nrm4 = 0
 * elsewhere). */
nsm_status nsm_gen_gbuffer(int H, int W, const float* cam, int n_obj, const float* objects, float* pos4,
                           float* nrm4, uint8_t* mask, void* stream);

/* lcam (host, 13 floats): emitter centre L[3], forward[3], right[3], up[3],
 * tan(fov / 2).  depth [Hs][Ws]: distance from L to the nearest hit along the
 * ray through texel (i, j)'s centre (ndc 2 (i + 1/2) / Ws - 1, 2 (j + 1/2) /
 * Hs - 1, row 0 at ndc_y = -1), z_far where nothing is hit before z_far. */
nsm_status nsm_gen_shadowmap(int Hs, int Ws, const float* lcam, float z_far, int n_obj, const float* objects,
                             float* depth, void* stream);

/* Monte-Carlo visibility of a spherical emitter (centre light_pos (host, 3
 * floats), radius) seen as its silhouette disk perpendicular to L - P:
 * spp_side^2 stratified jittered samples per pixel (SplitMix64 jitter keyed by
 * seed, pixel and sample), concentric disk map, shadow rays from P + eps n;
 * vis [H][W] float = unoccluded fraction, 1 where mask is 0.  radius 0 gives
 * the hard (point-light) visibility.  pos4 / nrm4 / mask as written by
 * nsm_gen_gbuffer. */
nsm_status nsm_gen_visibility(int H, int W, const float* pos4, const float* nrm4, const uint8_t* mask,
                              const float* light_pos, float radius, int spp_side, uint64_t seed, float eps,
                              int n_obj, const float* objects, float* vis, void* stream);

/* ---------------------------------------------------------------- deeper networks */

/* The encoder / decoder with L = 2 .. 7 levels (Sec. 3.6: the depth the 95th
 * percentile penumbra asks for; 3, 5 and 7 levels have receptive fields of
 * 24, 96 and 384 pixels), FP32 on CUDA cores.  Channel plan as for
 * three levels with widths 16 * 2^l (see nsm_param_count): for each layer in
 * the order enc0 3x3, enc0 1x1, ..., enc(L-2) 1x1, bottleneck 3x3, 1x1,
 * dec(L-2) 3x3, 1x1, ..., dec0 3x3, 1x1, head, its OIHW weights then bias.
 * nsm_param_count_levels: the vector's length (0 outside 2 .. 7; 39,521 for
 * 3 levels, 654,881 for 5).  nsm_infer_deep: visibility of a device frame
 * (H, W multiples of 2^(L-1), else NSM_ERR_SHAPE) from canonical FP32
 * parameters on the device; workspace (device, 256-byte aligned) of
 * nsm_infer_deep_workspace_bytes (84 floats per pixel plus one per parameter:
 * the weights re-laid out per call).  Asynchronous. */
size_t nsm_param_count_levels(int levels);
size_t nsm_infer_deep_workspace_bytes(int H, int W, int levels);
nsm_status nsm_infer_deep(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, int levels,
                          void* workspace, size_t workspace_bytes, float* vis_out, void* stream);

/* nsm_infer_deep with the form chosen: NSM_FP32 (exactly nsm_infer_deep),
 * NSM_FP8 (the three-term E4M3 form, 2 .. 7 levels: every 3x3 and 1x1 layer a
 * tcgen05 kind::f8f6f4 implicit GEMM over FP32 NHWC tensors, each activation
 * held as three E4M3 terms at fixed scales 1, 2^-4, 2^-8 and each weight of
 * output channel o as s_o times three such terms of W / s_o, s_o = max |W[o]| /
 * 448; the nine term products of a K step accumulate in FP32 in five blocks,
 * one per combined scale; activations above ~478 saturate; the head FP32 --
 * unlike nsm_infer's single-term NSM_FP8 form, within 1e-2 max-abs / 1e-4 MSE
 * of the FP64 network) or
 * NSM_BF16 (levels >= 3; NSM_ERR_UNSUPPORTED for 2): levels 0 and 1, whose
 * shapes are the 3-level network's, on its compensated-BF16 tensor-core stage
 * kernels (gather fused into the level-0 encoder, the level-0 decoder on the
 * coarse grid with the head), their weight images packed from this
 * network's vector (per call here; once with nsm_deep_weights below); every
 * 3x3 and 1x1 layer of levels 2 .. L-1 on a tcgen05 implicit GEMM over FP32
 * NHWC tensors with compensated BF16 operands (hi + lo
 * pairs, FP32 accumulation).  Workspace (device, 256-byte aligned) of
 * nsm_infer_deep_ex_workspace_bytes (0 for an unsupported combination).  A
 * bounded device wait that gives up sets the context's error word
 * (nsm_ctx_check).  Asynchronous. */
size_t nsm_infer_deep_ex_workspace_bytes(int H, int W, int levels, nsm_precision precision);
nsm_status nsm_infer_deep_ex(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, int levels,
                             nsm_precision precision, void* workspace, size_t workspace_bytes, float* vis_out,
                             void* stream);

/* Packed weights of an L-level network in one form, made once instead of per
 * call.  nsm_infer_deep_ex re-lays the weights out in its workspace on every
 * call (FP32: tap-major transposition; BF16: the stage kernels' images and
 * the inner levels' tcgen05 images; FP8: the three-term E4M3 images and
 * per-channel scales); nsm_deep_weights holds a device copy of the canonical
 * vector and those images, so a serving loop pays neither the packing
 * kernels nor the images' workspace.
 *
 * nsm_deep_weights_create: host_params (host, n floats, n =
 * nsm_param_count_levels(levels), finite; read before return) copied to the
 * current device and packed for `precision` (FP32, BF16 with levels >= 3, or
 * FP8); synchronous; NSM_ERR_SHAPE for a wrong n, NSM_ERR_UNSUPPORTED for a
 * form the depth lacks, NSM_ERR_CUDA if an allocation fails (nothing is kept).
 * *out is owned by the caller until nsm_deep_weights_destroy (NULL is a no-op;
 * frees device memory: no call may be in flight with the weights).
 * nsm_deep_weights_load_device: replace the weights with dev_params (device,
 * same n) and re-pack, asynchronous on `stream`, on the device the weights were
 * made on (NSM_ERR_INVALID_ARG otherwise); the caller orders it after calls
 * that still read the old weights.
 * nsm_infer_deep_packed: nsm_infer_deep_ex from packed weights, bit-identical
 * to it for the same vector and form; workspace (device, 256-byte aligned) of
 * nsm_infer_deep_packed_workspace_bytes (0 for an unsupported combination;
 * the ex workspace less the images), on the device the weights were made on.
 * Asynchronous; the same error word as nsm_infer_deep_ex. */
typedef struct nsm_deep_weights nsm_deep_weights;
nsm_status nsm_deep_weights_create(nsm_ctx* ctx, const float* host_params, size_t n, int levels,
                                   nsm_precision precision, nsm_deep_weights** out);
nsm_status nsm_deep_weights_load_device(nsm_deep_weights* w, const float* dev_params, size_t n, void* stream);
void nsm_deep_weights_destroy(nsm_deep_weights* w);
size_t nsm_infer_deep_packed_workspace_bytes(int H, int W, int levels, nsm_precision precision);
nsm_status nsm_infer_deep_packed(nsm_ctx* ctx, const nsm_frame* frame, const nsm_deep_weights* w, void* workspace,
                                 size_t workspace_bytes, float* vis_out, void* stream);

/* ---------------------------------------------------------------- frame analysis */

/* Temporal instability (Sec. 3.4, Eq. 3) of one pair of consecutive frames:
 * adds sum over accepted pixels p of exp(alpha D(p)) - 1, D(p) = |vis(p) -
 * vis_prev(m(p))|, to *sum_inout and the number of accepted pixels to
 * *count_inout (both device, accumulated so that a sequence sums over its
 * pairs; E = sum / (H W (T - 1)), alpha = 3 in the paper).  m(p): the world
 * position pos4(p).xyz projected with the previous frame's pinhole camera
 * cam_prev (host, 14 floats as in nsm_gen_gbuffer), nearest pixel.  p is
 * accepted iff pos4(p).w > 0, the projection is in front of the camera and
 * inside the image, pos4_prev(m).w > 0, |pos4_prev(m).w - z| <= 0.01 z (z the
 * reprojected view depth) and n(p) . n_prev(m) >= 0.9.  Reprojection, the
 * tests and D are binary32 with a fixed operation order (no contraction);
 * exp(alpha D) - 1 is evaluated in binary32 and summed in binary64.
 * vis / vis_prev [H][W] float; pos4 / nrm4 / pos4_prev / nrm4_prev [H][W]
 * float4 as written by nsm_gen_gbuffer (device). */
nsm_status nsm_temporal_instability(int H, int W, const float* vis, const float* vis_prev, const float* pos4,
                                    const float* nrm4, const float* pos4_prev, const float* nrm4_prev,
                                    const float* cam_prev, float alpha, double* sum_inout,
                                    unsigned long long* count_inout, void* stream);

#define NSM_MAX_PENUMBRA_BINS 8192

/* Histogram of screen-space penumbra widths (Sec. 3.6): for every pixel with a
 * blocker (blocker_out channel 1, z_max, > 0, as written by nsm_features) and
 * view depth d = pos4.w > 0, w = width H / (2 d tan_half_fovy) pixels (width =
 * blocker_out channel 2), counted in bin floor(w / bin_px) of hist_inout
 * (device, nbins uint32, accumulated; negative widths in bin 0, the last bin
 * open-ended).  binary32 arithmetic.  1 <= nbins <= NSM_MAX_PENUMBRA_BINS. */
nsm_status nsm_penumbra_histogram(int H, int W, const float* blocker, const float* pos4, float tan_half_fovy,
                                  float bin_px, int nbins, uint32_t* hist_inout, void* stream);

/* Depth from a penumbra histogram (Sec. 3.6), host only: *p95_px = upper edge
 * of the first bin at which the cumulative count reaches 95% of the total
 * (exactly: 20 cum >= 19 total; 0 for an empty histogram) and *levels = the
 * smallest l >= 1 with a receptive field 3 * 2^l >= *p95_px, i.e.
 * ceil(log2(p95 / 3)). */
nsm_status nsm_depth_for_penumbra(const uint32_t* hist, int nbins, float bin_px, float* p95_px, int* levels);

/* ---------------------------------------------------------------- feature sensitivity (Sec. 3.2, Eq. 1) */

/* Per-channel sums of the four input features over the frame's pixels, added
 * to moments_inout (device, 8 doubles: sum f_0..f_3, then sum f_0^2..f_3^2),
 * for the standard deviation sigma_i of each channel over a set of frames
 * (the paper estimates it over all pixels of its dataset).  H, W any size.
 * Asynchronous on stream. */
nsm_status nsm_feature_moments(const nsm_frame* frame, double* moments_inout, void* stream);

/* Workspace bytes of nsm_sensitivity for an H x W view (0 if invalid). */
size_t nsm_sensitivity_workspace_bytes(int H, int W);

/* Sensitivity of the network output to each input feature channel (Eq. 1):
 * one base inference and, for every channel i and draw k, one inference with
 * feature channel i perturbed by eps = 0.1 sigma[i] noise[k][i][p] inside the
 * gather; adds sum_p |phi_pert(p) - phi(p)| / (0.1 sigma[i]) to s_inout[i]
 * (device, 4 doubles).  Dividing by the number of pixels and draws gives
 * S_i = E|phi(f_i + eps_i) - phi(f_i)| / (0.1 sigma_i); s_i = S_i / sum S the
 * relative sensitivity.  Reading: Eq. 1's expectation is taken of the
 * absolute change (the signed change averages to about zero for symmetric
 * noise); eps_i has standard deviation 0.1 sigma_i.
 *   noise      device, [draws][4][H][W] floats: the caller's standard normal
 *              draws (the method's random numbers are inputs)
 *   sigma      host, 4 floats > 0
 *   precision  NSM_FP32 or NSM_BF16 (3-level weights); others NSM_ERR_UNSUPPORTED
 *   workspace  device, nsm_sensitivity_workspace_bytes(H, W), 256-byte aligned
 * H, W multiples of 4.  1 + 4 draws inference passes.  Asynchronous on stream. */
nsm_status nsm_sensitivity(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* weights, nsm_precision precision,
                           const float* noise, int draws, const float* sigma, void* workspace, size_t workspace_bytes,
                           double* s_inout, void* stream);

/* ---------------------------------------------------------------- no-allocation variant */

/* FP32 inference that allocates nothing and needs no workspace, for callers
 * that hold only their own input and output buffers and may not allocate
 * device memory (e.g. a per-frame render loop or a plug-in whose host engine
 * forbids device allocation after start-up, since an allocation can
 * synchronise the device and stall a frame).  The paper has no counterpart:
 * this is a deployment convenience of this library.
 *   dev_params  device, the canonical FP32 parameter vector (nsm_param_count
 *               floats, layout as for nsm_weights_create).
 *   vis_out     device, H*W floats.
 * Same results as nsm_infer with NSM_FP32.  The activations live in one fixed
 * device array inside the library, sized for H * W <= 262,144 pixels (e.g.
 * 512 x 512; about 21 MB, held on every device that loads the library until
 * the process exits); larger views return NSM_ERR_SHAPE.  Every call shares
 * that array: calls whose work overlaps on the GPU race and must be ordered by
 * the caller (one stream, or events).  Every call looks up the array's
 * device address in the current context (a host-side lookup that allocates
 * nothing); the first call in a context may load the library's device code,
 * so make it before any stream capture.
 * Errors: the frame checks of nsm_infer (NULL frame, sizes, H and W multiples
 * of 4, finite light / camera values, radius and bias >= 0, tan_half_fov > 0,
 * device pointers of the current device) give NSM_ERR_INVALID_ARG /
 * NSM_ERR_SHAPE / NSM_ERR_ALIGNMENT before any work; so does a buffer whose
 * allocation is shorter than it must be (dev_params nsm_param_count floats,
 * vis_out H*W floats, pos4 / nrm4 H*W float4, sm Hs*Ws floats).
 * Asynchronous on stream. */
nsm_status nsm_infer_fp32_static(const nsm_frame* frame, const float* dev_params, float* vis_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NSM_H */
