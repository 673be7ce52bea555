// C ABI of the backward and training entry points (include/nsm.h).
#include <vector>

#include <cuda_bf16.h>

#include "nsm_internal.h"
#include "train_internal.h"
#include "ctx_internal.h"
#include "tc_stage.h"

struct nsm_train_state {
    int device;
    int max_B, max_T, H, W;
    size_t n;            // parameters
    float* theta;        // FP32 master weights
    float* m;            // Adam first moment
    float* v;            // Adam second moment
    float* grad;         // gradient of the last step
    float* loss;         // device scalar
    nsm::GatherParams* gp;  // per-instance gather parameters (device)
    float* work;         // FP32 workspace
    int step;
    // Forward of the detached instances x_i (i >= 1) of Eq. 2: NSM_FP32 (the
    // checkpointed FP32 kernels, default) or NSM_BF16 (the tensor-core stage
    // kernels, BF16 images of the master weights packed every step)
    int detached_precision;
    // Forward of the target instances x_0 (the backward's checkpoints): NSM_FP32
    // (default) or NSM_BF16 (the stage kernels; their BF16-pair checkpoints
    // converted to FP32 for the FP32 backward)
    int forward_precision;
    // 3x3 recomputations and data gradients of the backward: NSM_FP32 (default)
    // or NSM_BF16 (tcgen05, compensated BF16 operands, FP32 accumulation)
    int backward_precision;
    uint4* conv3;        // their weight images, packed every step
    uint16_t* bf16;      // packed BF16 weight images
    void* descs;         // their packing table (device)
    int ndesc;
    int last_N;          // instances of the last nsm_train_grad call
};

namespace nsm {

static size_t backward_floats(int H, int W) { return tr::workspace_floats(1, 1, H, W); }
static size_t conv3_image_bytes() {
    return align_up(static_cast<size_t>(tr::conv3_images().total_chunks) * sizeof(uint4), 256);
}

// In place: n pixels of BF16 hi + lo pairs [pixel][part][C] -> FP32 [pixel][C]
// (same bytes per pixel; each thread reads a whole pixel before writing it).
template <int C>
__global__ void pairs_to_f32_kernel(void* buf, size_t n) {
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        uint4* px = static_cast<uint4*>(buf) + p * (C / 4);
        uint4 c[C / 4];
#pragma unroll
        for (int k = 0; k < C / 4; ++k) c[k] = px[k];
        const uint16_t* h = reinterpret_cast<const uint16_t*>(c);
        float f[C];
#pragma unroll
        for (int k = 0; k < C; ++k)
            f[k] = __bfloat162float(__ushort_as_bfloat16(h[k])) + __bfloat162float(__ushort_as_bfloat16(h[C + k]));
#pragma unroll
        for (int k = 0; k < C / 4; ++k) px[k] = make_uint4(__float_as_uint(f[4 * k]), __float_as_uint(f[4 * k + 1]),
                                                            __float_as_uint(f[4 * k + 2]), __float_as_uint(f[4 * k + 3]));
    }
}

template <int C>
static cudaError_t pairs_to_f32(float* buf, size_t n, cudaStream_t st) {
    const size_t blocks = (n + 255) / 256;
    pairs_to_f32_kernel<C><<<static_cast<int>(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(buf, n);
    return cudaGetLastError();
}

// The network on the tensor-core stage kernels for instances [i0, i1): gather
// fused, activations in the instances' checkpoint slots, visibility in b.vis.
static cudaError_t tc_forward(nsm_ctx* ctx, const nsm_train_state* s, const std::vector<GatherParams>& gps,
                              const tr::Buffers& b, int i0, int i1, size_t npx, cudaStream_t cs) {
    const size_t p1 = npx / 4, p2 = npx / 16;
    for (int j0 = i0; j0 < i1; j0 += kMaxViews) {
        const int n = (i1 - j0) < kMaxViews ? (i1 - j0) : kMaxViews;
        std::vector<Activations> act(n);
        std::vector<float*> vis(n);
        for (int k = 0; k < n; ++k) {
            const size_t i = static_cast<size_t>(j0 + k);
            act[k].e0 = b.e0 + i * p1 * 16;
            act[k].s1 = b.s1 + i * p1 * 32;
            act[k].p1 = b.p1 + i * p2 * 32;
            act[k].bo = b.bo + i * p2 * 32;
            act[k].d1 = b.d1 + i * p1 * 16;
            vis[k] = b.vis + i * npx;
        }
        TcBatch tb[kTcStages];
        tc_make_batches(gps.data() + j0, act.data(), vis.data(), n, s->theta, s->bf16, ctx->d_err, tb);
        for (int k = 0; k < kTcStages; ++k) {
            cudaError_t e = tc_launch_stage(k, ctx->tc_variant[k], tb[k], ctx->tc_ctas[k], cs);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace nsm

using namespace nsm;

extern "C" {

size_t nsm_backward_workspace_bytes(int H, int W) {
    if (H <= 0 || W <= 0) return 0;
    return align_up(sizeof(GatherParams), 256) + conv3_image_bytes() + backward_floats(H, W) * sizeof(float);
}

nsm_status nsm_backward(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, const float* grad_vis,
                        float* grad_params, float* grad_feat, float* vis_out, void* workspace,
                        size_t workspace_bytes, void* stream) {
    return nsm_backward_ex(ctx, frame, dev_params, grad_vis, grad_params, grad_feat, vis_out, NSM_FP32, workspace,
                           workspace_bytes, stream);
}

nsm_status nsm_backward_ex(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, const float* grad_vis,
                           float* grad_params, float* grad_feat, float* vis_out, nsm_precision precision,
                           void* workspace, size_t workspace_bytes, void* stream) {
    if (!ctx) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    if (precision != NSM_FP32 && precision != NSM_BF16)
        return fail(NSM_ERR_UNSUPPORTED, "the backward's 3x3 layers run in the FP32 or the BF16 form");
    nsm_status s = check_frame(frame, true);
    if (s != NSM_OK) return s;
    const int H = frame->H, W = frame->W;
    if (static_cast<size_t>(H) * W == 0) return NSM_OK;
    if ((s = check_dev_ptr(dev_params, "dev_params", 4)) != NSM_OK) return s;
    if ((s = check_dev_ptr(grad_vis, "grad_vis", 4)) != NSM_OK) return s;
    if ((s = check_dev_ptr(grad_params, "grad_params", 4)) != NSM_OK) return s;
    if ((s = check_dev_ptr(grad_feat, "grad_feat", 4, true)) != NSM_OK) return s;
    if ((s = check_dev_ptr(vis_out, "vis_out", 4, true)) != NSM_OK) return s;
    const size_t need = nsm_backward_workspace_bytes(H, W);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GatherParams g = make_gather(frame);
    GatherParams* dgp = static_cast<GatherParams*>(workspace);
    uint4* img = reinterpret_cast<uint4*>(static_cast<char*>(workspace) + align_up(sizeof(GatherParams), 256));
    float* base = reinterpret_cast<float*>(reinterpret_cast<char*>(img) + conv3_image_bytes());
    cudaError_t e = cudaMemcpyAsync(dgp, &g, sizeof(g), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload gather parameters");
    tr::Buffers b = tr::carve(base, 1, 1, H, W);
    if ((e = tr::features_batch(dgp, 1, H, W, b.feat, st)) != cudaSuccess) return cuda_fail(e, "features");
    if ((e = tr::forward(dev_params, b, 1, 1, H, W, st)) != cudaSuccess) return cuda_fail(e, "forward");
    const size_t npx = static_cast<size_t>(H) * W;
    if ((e = cudaMemcpyAsync(b.gvis, grad_vis, npx * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy cotangent");
    if (vis_out && (e = cudaMemcpyAsync(vis_out, b.vis, npx * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy visibility");
    const bool tcb = precision == NSM_BF16;
    if (tcb && (e = tr::conv3_pack(dev_params, img, st)) != cudaSuccess) return cuda_fail(e, "pack 3x3 images");
    if ((e = tr::backward(dev_params, grad_params, b, 1, H, W, grad_feat, st, tcb ? img : nullptr, ctx->d_err)) !=
        cudaSuccess)
        return cuda_fail(e, "backward");
    return NSM_OK;
}

nsm_status nsm_train_state_create(nsm_ctx* ctx, const float* host_params, size_t n, int max_B, int max_T, int H,
                                  int W, nsm_train_state** out) {
    if (!ctx || !host_params || !out) return fail(NSM_ERR_INVALID_ARG, "ctx, host_params and out must be non-NULL");
    *out = nullptr;
    if (n != nsm_param_count()) return fail(NSM_ERR_SHAPE, "parameter vector has %zu floats, expected %zu", n, nsm_param_count());
    if (max_B < 1 || max_T < 1 || H < 4 || W < 4 || (H % 4) || (W % 4) || H > 4096 || W > 4096)
        return fail(NSM_ERR_SHAPE, "batch %d x %d of %d x %d crops not supported", max_B, max_T, H, W);
    if (!finite_all(host_params, static_cast<int>(n))) return fail(NSM_ERR_INVALID_ARG, "parameters must be finite");
    nsm_train_state* s = new nsm_train_state{};
    cudaGetDevice(&s->device);
    s->max_B = max_B; s->max_T = max_T; s->H = H; s->W = W; s->n = n;
    const int N = max_B * max_T;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    alloc(reinterpret_cast<void**>(&s->theta), n * 4);
    alloc(reinterpret_cast<void**>(&s->m), n * 4);
    alloc(reinterpret_cast<void**>(&s->v), n * 4);
    alloc(reinterpret_cast<void**>(&s->grad), n * 4);
    alloc(reinterpret_cast<void**>(&s->loss), 256);
    alloc(reinterpret_cast<void**>(&s->gp), sizeof(GatherParams) * N);
    alloc(reinterpret_cast<void**>(&s->work), tr::workspace_floats(N, max_B, H, W) * 4);
    const BF16Images im = bf16_images();
    s->ndesc = im.n;
    alloc(reinterpret_cast<void**>(&s->bf16), im.total * sizeof(uint16_t));
    alloc(&s->descs, pack_desc_bytes() * im.n);
    alloc(reinterpret_cast<void**>(&s->conv3), static_cast<size_t>(tr::conv3_images().total_chunks) * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMemcpy(s->descs, im.desc, pack_desc_bytes() * im.n, cudaMemcpyHostToDevice);
    s->detached_precision = NSM_FP32;
    s->forward_precision = NSM_FP32;
    s->backward_precision = NSM_FP32;
    if (e == cudaSuccess) e = cudaMemcpy(s->theta, host_params, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->m, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(s->v, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(s->grad, 0, n * 4);
    if (e != cudaSuccess) {
        nsm_train_state_destroy(s);
        return cuda_fail(e, "train state allocation");
    }
    *out = s;
    return NSM_OK;
}

void nsm_train_state_destroy(nsm_train_state* s) {
    if (!s) return;
    cudaFree(s->theta); cudaFree(s->m); cudaFree(s->v); cudaFree(s->grad);
    cudaFree(s->loss); cudaFree(s->gp); cudaFree(s->work);
    cudaFree(s->bf16); cudaFree(s->descs); cudaFree(s->conv3);
    delete s;
}

static bool cfg_ok(const nsm_train_cfg* cfg) {
    return cfg->lr > 0.f && cfg->alpha >= 0.f && cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f &&
           cfg->beta2 < 1.f && cfg->eps > 0.f;
}

nsm_status nsm_train_grad(nsm_ctx* ctx, nsm_train_state* s, const nsm_batch* bt, const nsm_train_cfg* cfg,
                          float* loss_out, void* stream) {
    if (!ctx || !s || !bt || !cfg) return fail(NSM_ERR_INVALID_ARG, "ctx, state, batch and cfg must be non-NULL");
    if (bt->B < 1 || bt->T < 1 || bt->B > s->max_B || bt->T > s->max_T || bt->H != s->H || bt->W != s->W)
        return fail(NSM_ERR_SHAPE, "batch %d x %d of %d x %d does not fit the state (%d x %d of %d x %d)", bt->B,
                    bt->T, bt->H, bt->W, s->max_B, s->max_T, s->H, s->W);
    if (bt->Hs < 1 || bt->Ws < 1 || bt->Hs > 16384 || bt->Ws > 16384) return fail(NSM_ERR_SHAPE, "bad shadow-map size");
    if (!bt->lights || !bt->cameras) return fail(NSM_ERR_INVALID_ARG, "lights / cameras are NULL");
    if (!cfg_ok(cfg)) return fail(NSM_ERR_INVALID_ARG, "bad training configuration");
    nsm_status st;
    if ((st = check_dev_ptr(bt->pos4, "batch.pos4", 16)) != NSM_OK) return st;
    if ((st = check_dev_ptr(bt->nrm4, "batch.nrm4", 16)) != NSM_OK) return st;
    if ((st = check_dev_ptr(bt->sm, "batch.sm", 4)) != NSM_OK) return st;
    if ((st = check_dev_ptr(bt->target, "batch.target", 4)) != NSM_OK) return st;
    if ((st = check_dev_ptr(loss_out, "loss_out", 4, true)) != NSM_OK) return st;
    const int N = bt->B * bt->T, H = bt->H, W = bt->W;
    const size_t npx = static_cast<size_t>(H) * W;
    std::vector<GatherParams> gps(N);
    for (int i = 0; i < N; ++i) {
        nsm_frame f{};
        f.H = H; f.W = W; f.Hs = bt->Hs; f.Ws = bt->Ws;
        f.pos4 = bt->pos4 + static_cast<size_t>(i) * npx * 4;
        f.nrm4 = bt->nrm4 + static_cast<size_t>(i) * npx * 4;
        f.sm = bt->sm + static_cast<size_t>(i) * bt->Hs * bt->Ws;
        f.light = bt->lights[i];
        f.camera = bt->cameras[i];
        if (!finite_all(f.light.view_proj, 16) || !finite_all(f.light.pos, 3) || !finite_all(f.camera.pos, 3))
            return fail(NSM_ERR_INVALID_ARG, "instance %d: light / camera must be finite", i);
        gps[i] = make_gather(&f);
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(s->gp, gps.data(), sizeof(GatherParams) * N, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "upload gather parameters");
    tr::Buffers b = tr::carve(s->work, N, bt->B, H, W);
    s->last_N = N;
    const int B = bt->B;
    const bool tc0 = s->forward_precision == NSM_BF16;                   // x_0 on the tensor cores
    const bool tcd = s->detached_precision == NSM_BF16 && bt->T > 1;     // x_1 .. x_{T-1} on the tensor cores
    // features of the instances the FP32 kernels run, and of every x_0 (the
    // backward recomputes its first level from them)
    const int nfeat = tcd ? B : N;
    if ((e = tr::features_batch(s->gp, nfeat, H, W, b.feat, cs)) != cudaSuccess) return cuda_fail(e, "features");
    if (tc0 || tcd) {
        if ((e = launch_pack_bf16(s->theta, s->bf16, s->descs, s->ndesc, cs)) != cudaSuccess)
            return cuda_fail(e, "pack BF16 weights");
    }
    if (!tc0) {
        // x_0 (and, unless they run on the tensor cores, the detached instances) in FP32
        if ((e = tr::forward(s->theta, b, tcd ? B : N, B, H, W, cs)) != cudaSuccess) return cuda_fail(e, "forward");
    } else {
        if ((e = tc_forward(ctx, s, gps, b, 0, B, npx, cs)) != cudaSuccess) return cuda_fail(e, "forward (tensor cores)");
        // the FP32 backward reads FP32 checkpoints: e0, p1 and d1 were stored as BF16 pairs
        const size_t p1 = npx / 4, p2 = npx / 16;
        if ((e = pairs_to_f32<16>(b.e0, B * p1, cs)) != cudaSuccess ||
            (e = pairs_to_f32<32>(b.p1, B * p2, cs)) != cudaSuccess ||
            (e = pairs_to_f32<16>(b.d1, B * p1, cs)) != cudaSuccess)
            return cuda_fail(e, "checkpoint conversion");
        if (!tcd && bt->T > 1) {
            // detached instances in FP32: the fused forward over instances B .. N-1
            tr::Buffers bd = b;
            bd.feat += static_cast<size_t>(B) * npx * 4; bd.e0 += B * p1 * 16; bd.s1 += B * p1 * 32;
            bd.p1 += B * p2 * 32; bd.bo += B * p2 * 32; bd.d1 += B * p1 * 16; bd.vis += static_cast<size_t>(B) * npx;
            if ((e = tr::forward(s->theta, bd, N - B, B, H, W, cs)) != cudaSuccess) return cuda_fail(e, "forward");
        }
    }
    if (tcd && (e = tc_forward(ctx, s, gps, b, B, N, npx, cs)) != cudaSuccess)
        return cuda_fail(e, "detached forward (tensor cores)");
    if ((e = cudaMemsetAsync(s->loss, 0, sizeof(float), cs)) != cudaSuccess) return cuda_fail(e, "loss reset");
    if ((e = tr::loss_l1(b.vis, bt->target, bt->B, bt->T, npx, cfg->alpha, b.gvis, s->loss, cs)) != cudaSuccess)
        return cuda_fail(e, "loss");
    if ((e = cudaMemsetAsync(s->grad, 0, s->n * 4, cs)) != cudaSuccess) return cuda_fail(e, "grad reset");
    const bool tcb = s->backward_precision == NSM_BF16;
    if (tcb && (e = tr::conv3_pack(s->theta, s->conv3, cs)) != cudaSuccess) return cuda_fail(e, "pack 3x3 images");
    if ((e = tr::backward(s->theta, s->grad, b, bt->B, H, W, nullptr, cs, tcb ? s->conv3 : nullptr, ctx->d_err)) !=
        cudaSuccess)
        return cuda_fail(e, "backward");
    if (loss_out && (e = cudaMemcpyAsync(loss_out, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, cs)) != cudaSuccess)
        return cuda_fail(e, "copy loss");
    return NSM_OK;
}

nsm_status nsm_train_apply(nsm_ctx* ctx, nsm_train_state* s, const nsm_train_cfg* cfg, void* stream) {
    if (!ctx || !s || !cfg) return fail(NSM_ERR_INVALID_ARG, "ctx, state and cfg must be non-NULL");
    if (!cfg_ok(cfg)) return fail(NSM_ERR_INVALID_ARG, "bad training configuration");
    s->step += 1;
    const cudaError_t e = tr::adam(s->theta, s->grad, s->m, s->v, s->n, cfg->lr, cfg->beta1, cfg->beta2, cfg->eps,
                                   s->step, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "adam");
}

nsm_status nsm_train_step(nsm_ctx* ctx, nsm_train_state* s, const nsm_batch* bt, const nsm_train_cfg* cfg,
                          float* loss_out, void* stream) {
    const nsm_status st = nsm_train_grad(ctx, s, bt, cfg, loss_out, stream);
    return st != NSM_OK ? st : nsm_train_apply(ctx, s, cfg, stream);
}

nsm_status nsm_train_state_write(nsm_train_state* s, int what, const float* dev_in, size_t n, void* stream) {
    if (!s) return fail(NSM_ERR_INVALID_ARG, "state is NULL");
    if (n != s->n) return fail(NSM_ERR_SHAPE, "%zu floats given, the state holds %zu", n, s->n);
    nsm_status st = check_dev_ptr(dev_in, "dev_in", 4);
    if (st != NSM_OK) return st;
    float* dst = what == 0 ? s->theta : what == 1 ? s->grad : what == 2 ? s->m : what == 3 ? s->v : nullptr;
    if (!dst) return fail(NSM_ERR_INVALID_ARG, "unknown state vector %d", what);
    cudaError_t e = cudaMemcpyAsync(dst, dev_in, n * 4, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "copy state");
}

nsm_status nsm_train_state_set_detached_precision(nsm_train_state* s, nsm_precision precision) {
    if (!s) return fail(NSM_ERR_INVALID_ARG, "state is NULL");
    if (precision != NSM_FP32 && precision != NSM_BF16)
        return fail(NSM_ERR_UNSUPPORTED, "the detached instances run in the FP32 or the BF16 form");
    s->detached_precision = precision;
    return NSM_OK;
}

nsm_status nsm_train_state_set_forward_precision(nsm_train_state* s, nsm_precision precision) {
    if (!s) return fail(NSM_ERR_INVALID_ARG, "state is NULL");
    if (precision != NSM_FP32 && precision != NSM_BF16)
        return fail(NSM_ERR_UNSUPPORTED, "the target instances run in the FP32 or the BF16 form");
    s->forward_precision = precision;
    return NSM_OK;
}

nsm_status nsm_train_state_set_backward_precision(nsm_train_state* s, nsm_precision precision) {
    if (!s) return fail(NSM_ERR_INVALID_ARG, "state is NULL");
    if (precision != NSM_FP32 && precision != NSM_BF16)
        return fail(NSM_ERR_UNSUPPORTED, "the backward's 3x3 layers run in the FP32 or the BF16 form");
    s->backward_precision = precision;
    return NSM_OK;
}

nsm_status nsm_train_state_read_vis(nsm_train_state* s, float* dev_out, size_t n, void* stream) {
    if (!s) return fail(NSM_ERR_INVALID_ARG, "state is NULL");
    const size_t npx = static_cast<size_t>(s->H) * s->W;
    if (s->last_N < 1) return fail(NSM_ERR_INVALID_ARG, "no training step has run on this state");
    if (n != s->last_N * npx) return fail(NSM_ERR_SHAPE, "%zu floats requested, the last step has %zu", n, s->last_N * npx);
    nsm_status st = check_dev_ptr(dev_out, "dev_out", 4);
    if (st != NSM_OK) return st;
    const tr::Buffers b = tr::carve(s->work, s->last_N, s->max_B, s->H, s->W);
    cudaError_t e = cudaMemcpyAsync(dev_out, b.vis, n * 4, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "copy visibility");
}

nsm_status nsm_train_state_read(nsm_train_state* s, int what, float* dev_out, size_t n, void* stream) {
    if (!s) return fail(NSM_ERR_INVALID_ARG, "state is NULL");
    if (n != s->n) return fail(NSM_ERR_SHAPE, "%zu floats requested, the state holds %zu", n, s->n);
    nsm_status st = check_dev_ptr(dev_out, "dev_out", 4);
    if (st != NSM_OK) return st;
    const float* src = what == 0 ? s->theta : what == 1 ? s->grad : what == 2 ? s->m : what == 3 ? s->v : nullptr;
    if (!src) return fail(NSM_ERR_INVALID_ARG, "unknown state vector %d", what);
    cudaError_t e = cudaMemcpyAsync(dev_out, src, n * 4, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "copy state");
    return NSM_OK;
}

}  // extern "C"
