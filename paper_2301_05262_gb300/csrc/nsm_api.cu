#include <algorithm>
// C ABI of the library (include/nsm.h): argument validation, weight upload,
// workspace carving and dispatch to the kernels.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nsm.h"
#include "nsm_internal.h"

#include "ctx_internal.h"



namespace nsm {

static thread_local std::string g_last_error;

nsm_status fail(nsm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

nsm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(NSM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

LayerOffsets layer_offsets() {
    LayerOffsets o{};
    size_t off = 0;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        o.w[l] = off;
        off += static_cast<size_t>(kLayers[l].cin) * kLayers[l].cout * kLayers[l].k * kLayers[l].k;
        o.b[l] = off;
        off += kLayers[l].cout;
    }
    o.total = off;
    return o;
}

LayerOffsets layer_offsets_s2d() {
    LayerOffsets o{};
    size_t off = 0;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        if (l == ENC0_3 || l == ENC0_1 || l == DEC0_3 || l == DEC0_1) {
            o.w[l] = o.b[l] = SIZE_MAX;
            continue;
        }
        const int cout = l == HEAD ? kS2dHeadOut : kLayers[l].cout;
        o.w[l] = off;
        off += static_cast<size_t>(kLayers[l].cin) * cout * kLayers[l].k * kLayers[l].k;
        o.b[l] = off;
        off += cout;
    }
    o.total = off;
    return o;
}

// A memory pool owned by the library, one per device, for scratch buffers that
// live only for the kernels of one call (allocated and freed in stream order).
// It keeps up to 512 MiB mapped between calls, so a per-frame caller does not
// map and unmap pages every frame; the device's default pool is left alone.
cudaError_t scratch_pool(cudaMemPool_t* out) {
    static std::mutex m;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(m);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        if ((e = cudaMemPoolCreate(&p, &props)) != cudaSuccess) return e;
        uint64_t keep = 512ull << 20;
        if ((e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        pools[dev] = p;
    }
    *out = pools[dev];
    return cudaSuccess;
}

int resident_ctas_per_sm(const void* func, int threads, size_t dyn_smem) {
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0;
    if (cudaFuncGetAttributes(&fa, func) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess)
        return 1;
    const size_t smem = dyn_smem + fa.sharedSizeBytes + static_cast<size_t>(resv);
    const int warps = (threads + 31) / 32;
    // registers are allocated per warp in units of 256 (8 per thread, rounded up)
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int n = blk_sm;
    if (smem > 0) n = std::min<long long>(n, static_cast<long long>(smem_sm) / static_cast<long long>(smem));
    if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
    n = std::min(n, thr_sm / (32 * warps));
    return n < 1 ? 1 : n;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t activations_bytes(int H, int W, size_t eb, Activations* carve, void* base) {
    const size_t h2 = static_cast<size_t>(H / 2) * (W / 2), h4 = static_cast<size_t>(H / 4) * (W / 4);
    const size_t sizes[5] = {h2 * 16 * eb, h2 * 32 * eb, h4 * 32 * eb, h4 * 32 * eb, h2 * 16 * eb};
    size_t off = 0;
    void* ptrs[5];
    for (int i = 0; i < 5; ++i) {
        ptrs[i] = base ? static_cast<char*>(base) + off : nullptr;
        off += align_up(sizes[i], 256);
    }
    if (carve) { carve->e0 = ptrs[0]; carve->s1 = ptrs[1]; carve->p1 = ptrs[2]; carve->bo = ptrs[3]; carve->d1 = ptrs[4]; }
    return off;
}

// ------------------------------------------------------------------ checks
nsm_status check_device() {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(NSM_ERR_DEVICE, "no CUDA device: %s", cudaGetErrorString(e));
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3)
        return fail(NSM_ERR_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a only", dev, major, minor);
    return NSM_OK;
}

nsm_status check_dev_ptr(const void* p, const char* name, size_t align, bool nullable) {
    if (!p) {
        if (nullable) return NSM_OK;
        return fail(NSM_ERR_INVALID_ARG, "%s is NULL", name);
    }
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NSM_ERR_INVALID_ARG, "%s: cannot query pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(NSM_ERR_INVALID_ARG, "%s is not device memory", name);
    int dev = -1;
    cudaGetDevice(&dev);
    if (at.device != dev) return fail(NSM_ERR_INVALID_ARG, "%s lives on device %d, current device is %d", name, at.device, dev);
    if (reinterpret_cast<uintptr_t>(p) % align)
        return fail(NSM_ERR_ALIGNMENT, "%s must be %zu-byte aligned", name, align);
    return NSM_OK;
}

bool finite_all(const float* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!(v[i] == v[i]) || v[i] == INFINITY || v[i] == -INFINITY) return false;
    return true;
}

nsm_status check_frame_host(const nsm_frame* f, bool need_mult4) {
    if (!f) return fail(NSM_ERR_INVALID_ARG, "frame is NULL");
    if (f->H < 0 || f->W < 0 || f->H > 16384 || f->W > 16384)
        return fail(NSM_ERR_SHAPE, "view size %d x %d outside [0, 16384]", f->H, f->W);
    if (need_mult4 && ((f->H % 4) || (f->W % 4)))
        return fail(NSM_ERR_SHAPE, "view size %d x %d: H and W must be multiples of 4", f->H, f->W);
    if (f->Hs < 1 || f->Ws < 1 || f->Hs > 16384 || f->Ws > 16384)
        return fail(NSM_ERR_SHAPE, "shadow map %d x %d outside [1, 16384]", f->Hs, f->Ws);
    const nsm_light& l = f->light;
    if (!finite_all(l.pos, 3) || !finite_all(l.view_proj, 16) || !finite_all(f->camera.pos, 3) ||
        !finite_all(&l.radius, 1) || !finite_all(&l.r_hat, 1) || !finite_all(&l.z_far, 1) ||
        !finite_all(&l.bias, 1) || !finite_all(&l.tan_half_fov, 1))
        return fail(NSM_ERR_INVALID_ARG, "light / camera parameters must be finite");
    if (l.radius < 0.f || l.bias < 0.f || l.tan_half_fov <= 0.f)
        return fail(NSM_ERR_INVALID_ARG, "light radius and bias must be >= 0, tan_half_fov > 0");
    return NSM_OK;
}

nsm_status check_frame(const nsm_frame* f, bool need_mult4) {
    nsm_status s = check_frame_host(f, need_mult4);
    if (s != NSM_OK) return s;
    if (static_cast<size_t>(f->H) * f->W == 0) return NSM_OK;
    if ((s = check_dev_ptr(f->pos4, "frame.pos4", 16)) != NSM_OK) return s;
    if ((s = check_dev_ptr(f->nrm4, "frame.nrm4", 16)) != NSM_OK) return s;
    if ((s = check_dev_ptr(f->sm, "frame.sm", 4)) != NSM_OK) return s;
    return NSM_OK;
}

GatherParams make_gather(const nsm_frame* f) {
    GatherParams g{};
    std::memcpy(g.M, f->light.view_proj, sizeof(g.M));
    for (int k = 0; k < 3; ++k) { g.L[k] = f->light.pos[k]; g.C[k] = f->camera.pos[k]; }
    g.r_hat = f->light.r_hat;
    g.z_far = f->light.z_far;
    g.beta = f->light.bias;
    g.radius = f->light.radius;
    g.tan_half_fov = f->light.tan_half_fov;
    g.Ws = f->Ws; g.Hs = f->Hs;
    g.Ws_f = static_cast<float>(f->Ws); g.Hs_f = static_cast<float>(f->Hs);
    g.half_Ws = 0.5f * static_cast<float>(f->Ws);
    g.H = f->H; g.W = f->W;
    g.pos4 = reinterpret_cast<const float4*>(f->pos4);
    g.nrm4 = reinterpret_cast<const float4*>(f->nrm4);
    g.sm = f->sm;
    return g;
}

}  // namespace nsm

using namespace nsm;

// ====================================================================== C ABI
extern "C" {

int nsm_abi_version(void) { return NSM_ABI_VERSION; }

const char* nsm_last_error(void) { return g_last_error.c_str(); }

nsm_status nsm_ctx_create(nsm_ctx** out) {
    if (!out) return fail(NSM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    nsm_status s = check_device();
    if (s != NSM_OK) return s;
    nsm_ctx* c = new nsm_ctx{};
    cudaGetDevice(&c->device);
    for (int st = 0; st < kTcStages; ++st) { c->tc_variant[st] = tc_default_variant(st); c->tc_ctas[st] = 0; }
    cudaError_t e = cudaMalloc(&c->d_err, sizeof(int) * 4);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(error word)"); }
    e = cudaMemset(c->d_err, 0, sizeof(int) * 4);
    if (e != cudaSuccess) { cudaFree(c->d_err); delete c; return cuda_fail(e, "cudaMemset(error word)"); }
    *out = c;
    return NSM_OK;
}

void nsm_ctx_destroy(nsm_ctx* c) {
    if (!c) return;
    ctx_release_graph(c);
    ctx_release_host_slots(c);
    cudaFree(c->d_err);
    delete c;
}

nsm_status nsm_ctx_check(nsm_ctx* c) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int h[4] = {0, 0, 0, 0};
    e = cudaMemcpy(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read error word");
    if (h[0] != 0) {
        cudaMemset(c->d_err, 0, sizeof(h));
        return fail(NSM_ERR_TIMEOUT, "a bounded device wait gave up (code %d, site %d)", h[0], h[1]);
    }
    return NSM_OK;
}

nsm_status nsm_ctx_set_stage_events(nsm_ctx* c, void* const* events, int n) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !events)) return fail(NSM_ERR_INVALID_ARG, "bad event list");
    c->stage_events.clear();
    for (int i = 0; i < n; ++i) {
        if (!events[i]) return fail(NSM_ERR_INVALID_ARG, "event %d is NULL", i);
        c->stage_events.push_back(static_cast<cudaEvent_t>(events[i]));
    }
    return NSM_OK;
}

int nsm_infer_kernel_count(nsm_precision precision) {
    switch (precision) {
        case NSM_FP32: return kInferKernelsFp32;
        case NSM_BF16: return kInferKernelsBf16;
        case NSM_FP8: return kInferKernelsFp8;
        default: return 0;
    }
}

const char* nsm_infer_kernel_name(nsm_precision precision, int i) {
    if (i < 0 || i >= nsm_infer_kernel_count(precision)) return "";
    switch (precision) {
        case NSM_FP32: return kInferKernelNamesFp32[i];
        case NSM_BF16: return kInferKernelNamesBf16[i];
        case NSM_FP8: return kInferKernelNamesFp8[i];
        default: return "";
    }
}

size_t nsm_param_count(void) { return layer_offsets().total; }

size_t nsm_param_count_topology(nsm_topology t) {
    return t == NSM_TOPO_LEVELS3 ? layer_offsets().total : (t == NSM_TOPO_S2D ? layer_offsets_s2d().total : 0);
}

nsm_status nsm_weights_create(nsm_ctx* ctx, const float* host_params, size_t n, nsm_weights** out) {
    return nsm_weights_create_topology(ctx, NSM_TOPO_LEVELS3, host_params, n, out);
}

nsm_status nsm_weights_create_topology(nsm_ctx* ctx, nsm_topology topology, const float* host_params, size_t n,
                                       nsm_weights** out) {
    if (!ctx || !host_params || !out) return fail(NSM_ERR_INVALID_ARG, "ctx, host_params and out must be non-NULL");
    *out = nullptr;
    if (topology != NSM_TOPO_LEVELS3 && topology != NSM_TOPO_S2D)
        return fail(NSM_ERR_INVALID_ARG, "unknown topology %d", static_cast<int>(topology));
    const bool s2d = topology == NSM_TOPO_S2D;
    const size_t want = nsm_param_count_topology(topology);
    if (n != want) return fail(NSM_ERR_SHAPE, "parameter vector has %zu floats, expected %zu", n, want);
    if (!finite_all(host_params, static_cast<int>(n))) return fail(NSM_ERR_INVALID_ARG, "parameters must be finite");
    nsm_weights* w = new nsm_weights{};
    w->topology = topology;
    cudaGetDevice(&w->device);
    cudaError_t e = cudaMalloc(&w->d_params, n * sizeof(float));
    if (e != cudaSuccess) { delete w; return cuda_fail(e, "cudaMalloc(weights)"); }
    e = cudaMemcpy(w->d_params, host_params, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(w->d_params); delete w; return cuda_fail(e, "upload weights"); }
    const BF16Images im = bf16_images(s2d);
    w->ndesc = im.n;
    e = cudaMalloc(&w->d_bf16, im.total * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&w->d_descs, pack_desc_bytes() * im.n);
    if (e == cudaSuccess) e = cudaMemcpy(w->d_descs, im.desc, pack_desc_bytes() * im.n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_pack_bf16(w->d_params, w->d_bf16, w->d_descs, w->ndesc, nullptr);
    const F8Images f8 = fp8_images();
    if (!s2d) {
        if (e == cudaSuccess) e = cudaMalloc(&w->d_fp8, f8.img_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&w->d_fp8_scales, f8.scales * sizeof(float));
        if (e == cudaSuccess) e = launch_pack_fp8(w->d_params, w->d_fp8, w->d_fp8_scales, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(w->d_params); cudaFree(w->d_bf16); cudaFree(w->d_descs); cudaFree(w->d_fp8);
        cudaFree(w->d_fp8_scales); delete w;
        return cuda_fail(e, "pack weights");
    }
    *out = w;
    return NSM_OK;
}

nsm_status nsm_weights_load_device(nsm_weights* w, const float* dev_params, size_t n, void* stream) {
    if (!w) return fail(NSM_ERR_INVALID_ARG, "weights is NULL");
    const size_t want = nsm_param_count_topology(static_cast<nsm_topology>(w->topology));
    if (n != want) return fail(NSM_ERR_SHAPE, "parameter vector has %zu floats, expected %zu", n, want);
    nsm_status s = check_dev_ptr(dev_params, "dev_params", 4);
    if (s != NSM_OK) return s;
    cudaError_t e = cudaMemcpyAsync(w->d_params, dev_params, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "copy weights");
    e = launch_pack_bf16(w->d_params, w->d_bf16, w->d_descs, w->ndesc, static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess && w->topology == NSM_TOPO_LEVELS3)
        e = launch_pack_fp8(w->d_params, w->d_fp8, w->d_fp8_scales, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "pack weights");
    return NSM_OK;
}

void nsm_weights_destroy(nsm_weights* w) {
    if (!w) return;
    cudaFree(w->d_params);
    cudaFree(w->d_bf16);
    cudaFree(w->d_descs);
    cudaFree(w->d_fp8);
    cudaFree(w->d_fp8_scales);
    delete w;
}

static nsm_status features_impl(const nsm_frame* frame, float* feat_out, int32_t* texel_out, uint32_t* hard_out,
                                float* blocker_out, void* workspace, void* stream) {
    nsm_status s = check_frame(frame, false);
    if (s != NSM_OK) return s;
    if (static_cast<size_t>(frame->H) * frame->W == 0) return NSM_OK;
    if ((s = check_device()) != NSM_OK) return s;
    if ((s = check_dev_ptr(feat_out, "feat_out", 4)) != NSM_OK) return s;
    if ((s = check_dev_ptr(texel_out, "texel_out", 4, true)) != NSM_OK) return s;
    if ((s = check_dev_ptr(hard_out, "hard_out", 4, true)) != NSM_OK) return s;
    if ((s = check_dev_ptr(blocker_out, "blocker_out", 4, true)) != NSM_OK) return s;
    GatherParams g = make_gather(frame);
    cudaError_t e = launch_features(g, feat_out, texel_out, hard_out, blocker_out, workspace,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "features kernel launch");
    return NSM_OK;
}

nsm_status nsm_features(const nsm_frame* frame, float* feat_out, int32_t* texel_out, uint32_t* hard_out,
                        float* blocker_out, void* stream) {
    return features_impl(frame, feat_out, texel_out, hard_out, blocker_out, nullptr, stream);
}

size_t nsm_features_workspace_bytes(int Hs, int Ws) {
    if (Hs <= 0 || Ws <= 0) return 0;
    return static_cast<size_t>(Hs) * Ws * 16;
}

nsm_status nsm_features_ws(const nsm_frame* frame, float* feat_out, int32_t* texel_out, uint32_t* hard_out,
                           float* blocker_out, void* workspace, size_t workspace_bytes, void* stream) {
    if (blocker_out && frame && static_cast<size_t>(frame->H) * frame->W > 0) {
        const size_t need = nsm_features_workspace_bytes(frame->Hs, frame->Ws);
        if (!workspace || workspace_bytes < need)
            return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
        nsm_status s = check_dev_ptr(workspace, "workspace", 256);
        if (s != NSM_OK) return s;
    }
    return features_impl(frame, feat_out, texel_out, hard_out, blocker_out, blocker_out ? workspace : nullptr, stream);
}

size_t nsm_infer_workspace_bytes(int H, int W, nsm_precision precision) {
    if (H <= 0 || W <= 0) return 0;
    (void)precision;  // FP32 activations, or BF16 hi + lo pairs: 4 bytes per channel either way
    return activations_bytes(H, W, 4, nullptr, nullptr);
}

nsm_status nsm_infer(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w, nsm_precision precision,
                     void* workspace, size_t workspace_bytes, float* vis_out, void* stream) {
    return infer_impl(ctx, frame, w, precision, workspace, workspace_bytes, vis_out, stream, nullptr, 0.f, 0);
}

}  // extern "C"

namespace nsm {

nsm_status infer_impl(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w, nsm_precision precision,
                      void* workspace, size_t workspace_bytes, float* vis_out, void* stream, const float* feat_eps,
                      float eps_scale, int eps_ch) {
    if (!ctx) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    if (!w) return fail(NSM_ERR_INVALID_ARG, "weights is NULL");
    if (precision != NSM_FP32 && precision != NSM_BF16 && precision != NSM_FP8)
        return fail(NSM_ERR_INVALID_ARG, "unknown precision %d", static_cast<int>(precision));
    nsm_status s = check_frame(frame, true);
    if (s != NSM_OK) return s;
    if (static_cast<size_t>(frame->H) * frame->W == 0) return NSM_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != ctx->device || dev != w->device)
        return fail(NSM_ERR_DEVICE, "context / weights were created on another device");
    if ((s = check_dev_ptr(vis_out, "vis_out", 4)) != NSM_OK) return s;
    const size_t need = nsm_infer_workspace_bytes(frame->H, frame->W, precision);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    Activations act{};
    activations_bytes(frame->H, frame->W, 4, &act, workspace);
    GatherParams g = make_gather(frame);
    if (feat_eps) {
        if (w->topology != NSM_TOPO_LEVELS3 || (precision != NSM_FP32 && precision != NSM_BF16))
            return fail(NSM_ERR_UNSUPPORTED, "feature perturbations run in the 3-level FP32 and BF16 forms");
        g.feat_eps = feat_eps;
        g.eps_scale = eps_scale;
        g.eps_ch = eps_ch;
    }
    StageEvents se;
    const int k = nsm_infer_kernel_count(precision);
    if (!ctx->stage_events.empty()) {
        if (static_cast<int>(ctx->stage_events.size()) < k + 1)
            return fail(NSM_ERR_INVALID_ARG, "%zu stage events set, %d needed", ctx->stage_events.size(), k + 1);
        se.ev = ctx->stage_events.data();
        se.n = static_cast<int>(ctx->stage_events.size());
        se.stream = static_cast<cudaStream_t>(stream);
    }
    cudaError_t e;
    if (w->topology == NSM_TOPO_S2D) {
        if (precision != NSM_BF16)
            return fail(NSM_ERR_UNSUPPORTED, "space-to-depth weights run in the BF16 form only");
        e = launch_infer_s2d_bf16(g, w->d_params, w->d_bf16, act, vis_out, ctx->d_err,
                                  static_cast<cudaStream_t>(stream), se);
    } else if (precision == NSM_FP32)
        e = launch_infer_fp32(g, w->d_params, act, vis_out, static_cast<cudaStream_t>(stream), se);
    else if (precision == NSM_BF16)
        e = launch_infer_bf16(g, w->d_params, w->d_bf16, act, vis_out, ctx->d_err, static_cast<cudaStream_t>(stream), se,
                              ctx->tc_variant, ctx->tc_ctas);
    else
        e = launch_infer_fp8(g, w->d_params, w->d_fp8, w->d_fp8_scales, act, vis_out, ctx->d_err,
                             static_cast<cudaStream_t>(stream), se);
    if (e != cudaSuccess) return cuda_fail(e, "inference kernel launch");
    return NSM_OK;
}

}  // namespace nsm

extern "C" {

// Row slab of a frame: rows [y0, y1) computed from the sub-frame [sy0, sy1) =
// [y0 - halo, y1 + halo] clipped to the frame (every bound a multiple of 4,
// so the pooling grids of the slab and the frame coincide).
static void slab_bounds(int H, int y0, int y1, int halo, int* sy0, int* sy1) {
    *sy0 = y0 - halo < 0 ? 0 : y0 - halo;
    *sy1 = y1 + halo > H ? H : y1 + halo;
}

size_t nsm_infer_rows_workspace_bytes(int H, int W, int y0, int y1, int halo, nsm_precision precision) {
    if (H <= 0 || W <= 0 || y0 < 0 || y1 > H || y0 >= y1 || halo < 0) return 0;
    int sy0, sy1;
    slab_bounds(H, y0, y1, halo, &sy0, &sy1);
    const size_t hs = static_cast<size_t>(sy1 - sy0);
    return nsm_infer_workspace_bytes(static_cast<int>(hs), W, precision) + align_up(hs * W * sizeof(float), 256);
}

nsm_status nsm_infer_rows(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w, nsm_precision precision, int y0,
                          int y1, int halo, void* workspace, size_t workspace_bytes, float* vis_rows, void* stream) {
    nsm_status s = check_frame_host(frame, true);
    if (s != NSM_OK) return s;
    if (y0 < 0 || y1 > frame->H || y0 >= y1 || (y0 % 4) || (y1 % 4) || halo < 0 || (halo % 4))
        return fail(NSM_ERR_SHAPE, "rows [%d, %d) of %d with halo %d: bounds in the frame, multiples of 4", y0, y1,
                    frame->H, halo);
    if ((s = check_dev_ptr(vis_rows, "vis_rows", 4)) != NSM_OK) return s;
    const size_t need = nsm_infer_rows_workspace_bytes(frame->H, frame->W, y0, y1, halo, precision);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    int sy0, sy1;
    slab_bounds(frame->H, y0, y1, halo, &sy0, &sy1);
    nsm_frame sub = *frame;
    sub.H = sy1 - sy0;
    sub.pos4 = frame->pos4 + static_cast<size_t>(sy0) * frame->W * 4;
    sub.nrm4 = frame->nrm4 + static_cast<size_t>(sy0) * frame->W * 4;
    const size_t act = nsm_infer_workspace_bytes(sub.H, sub.W, precision);
    float* vis = reinterpret_cast<float*>(static_cast<char*>(workspace) + act);
    if ((s = infer_impl(ctx, &sub, w, precision, workspace, act, vis, stream, nullptr, 0.f, 0)) != NSM_OK) return s;
    const size_t W = static_cast<size_t>(frame->W);
    cudaError_t e = cudaMemcpyAsync(vis_rows, vis + static_cast<size_t>(y0 - sy0) * W,
                                    static_cast<size_t>(y1 - y0) * W * sizeof(float), cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "copy the slab's rows");
}

size_t nsm_infer_host_stage_bytes(int H, int W, int Hs, int Ws) {
    if (H <= 0 || W <= 0 || Hs <= 0 || Ws <= 0) return 0;
    const size_t npx = static_cast<size_t>(H) * W;
    return align_up(npx * 16, 256) * 2 + align_up(static_cast<size_t>(Hs) * Ws * 4, 256) + align_up(npx * 4, 256);
}

}  // extern "C"

// Copy streams and per-slot events of nsm_infer_host_sequence.
static nsm_status ctx_host_slots(nsm_ctx* c) {
    if (c->slots_ready) return NSM_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c->h2d_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking);
    for (int k = 0; k < kMaxHostSlots && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&c->slot_h2d[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->slot_inf[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->slot_d2h[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        c->slots_ready = true;  // release what was created
        ctx_release_host_slots(c);
        return cuda_fail(e, "copy streams / events");
    }
    c->slots_ready = true;
    return NSM_OK;
}

void ctx_release_host_slots(nsm_ctx* c) {
    if (!c->slots_ready) return;
    if (c->h2d_stream) cudaStreamDestroy(c->h2d_stream);
    if (c->d2h_stream) cudaStreamDestroy(c->d2h_stream);
    for (int k = 0; k < kMaxHostSlots; ++k) {
        if (c->slot_h2d[k]) cudaEventDestroy(c->slot_h2d[k]);
        if (c->slot_inf[k]) cudaEventDestroy(c->slot_inf[k]);
        if (c->slot_d2h[k]) cudaEventDestroy(c->slot_d2h[k]);
        c->slot_h2d[k] = c->slot_inf[k] = c->slot_d2h[k] = nullptr;
    }
    c->h2d_stream = c->d2h_stream = nullptr;
    c->slots_ready = false;
}

extern "C" {

nsm_status nsm_infer_host(nsm_ctx* ctx, const nsm_frame* hf, const nsm_weights* w, nsm_precision precision,
                          void* dev_stage, size_t stage_bytes, void* workspace, size_t workspace_bytes,
                          float* vis_host, void* stream) {
    if (!hf) return fail(NSM_ERR_INVALID_ARG, "frame is NULL");
    if (!hf->pos4 || !hf->nrm4 || !hf->sm || !vis_host)
        return fail(NSM_ERR_INVALID_ARG, "host pointers must be non-NULL");
    if (hf->H < 0 || hf->W < 0) return fail(NSM_ERR_SHAPE, "negative view size");
    const size_t npx = static_cast<size_t>(hf->H) * hf->W;
    if (npx == 0) return NSM_OK;
    const size_t need = nsm_infer_host_stage_bytes(hf->H, hf->W, hf->Hs, hf->Ws);
    if (!dev_stage || stage_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "staging buffer of %zu bytes given, %zu needed", stage_bytes, need);
    nsm_status s = check_dev_ptr(dev_stage, "dev_stage", 256);
    if (s != NSM_OK) return s;
    char* base = static_cast<char*>(dev_stage);
    float* d_pos = reinterpret_cast<float*>(base);
    float* d_nrm = reinterpret_cast<float*>(base + align_up(npx * 16, 256));
    float* d_sm = reinterpret_cast<float*>(base + 2 * align_up(npx * 16, 256));
    float* d_vis = reinterpret_cast<float*>(base + 2 * align_up(npx * 16, 256) +
                                            align_up(static_cast<size_t>(hf->Hs) * hf->Ws * 4, 256));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_pos, hf->pos4, npx * 16, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e, "H2D pos4");
    if ((e = cudaMemcpyAsync(d_nrm, hf->nrm4, npx * 16, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e, "H2D nrm4");
    if ((e = cudaMemcpyAsync(d_sm, hf->sm, static_cast<size_t>(hf->Hs) * hf->Ws * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "H2D shadow map");
    nsm_frame df = *hf;
    df.pos4 = d_pos; df.nrm4 = d_nrm; df.sm = d_sm;
    s = nsm_infer(ctx, &df, w, precision, workspace, workspace_bytes, d_vis, stream);
    if (s != NSM_OK) return s;
    if ((e = cudaMemcpyAsync(vis_host, d_vis, npx * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e, "D2H visibility");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return NSM_OK;
}

nsm_status nsm_infer_host_sequence(nsm_ctx* ctx, int n, const nsm_frame* frames, const nsm_weights* w,
                                   nsm_precision precision, void* dev_stage, size_t stage_bytes, void* workspace,
                                   size_t workspace_bytes, float* const* vis_host, void* stream) {
    if (!ctx || !w) return fail(NSM_ERR_INVALID_ARG, "ctx and weights must be non-NULL");
    if (n < 0 || (n > 0 && (!frames || !vis_host))) return fail(NSM_ERR_INVALID_ARG, "n >= 0, frames and vis_host");
    if (n == 0) return NSM_OK;
    size_t slot = 0;
    for (int i = 0; i < n; ++i) {
        const nsm_frame& f = frames[i];
        if (!f.pos4 || !f.nrm4 || !f.sm || !vis_host[i])
            return fail(NSM_ERR_INVALID_ARG, "frame %d: host pointers must be non-NULL", i);
        if (f.H < 0 || f.W < 0 || f.Hs <= 0 || f.Ws <= 0) return fail(NSM_ERR_SHAPE, "frame %d: bad sizes", i);
        const size_t b = nsm_infer_host_stage_bytes(f.H, f.W, f.Hs, f.Ws);
        if (b > slot) slot = b;
    }
    slot = align_up(slot, 256);
    const int nslots = slot ? static_cast<int>(stage_bytes / slot < kMaxHostSlots ? stage_bytes / slot : kMaxHostSlots)
                            : kMaxHostSlots;
    if (!dev_stage || nslots < 2)
        return fail(NSM_ERR_WORKSPACE, "staging buffer of %zu bytes given, 2 x %zu needed", stage_bytes, slot);
    nsm_status s = check_dev_ptr(dev_stage, "dev_stage", 256);
    if (s != NSM_OK) return s;
    if ((s = ctx_host_slots(ctx)) != NSM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream), cs = ctx->h2d_stream, ds = ctx->d2h_stream;
    cudaError_t e = cudaSuccess;
    // slot k's buffers are free again once the read-back of the frame that used
    // them is done (which itself waited for that frame's inference)
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const int k = i % nslots;
        const nsm_frame& hf = frames[i];
        const size_t npx = static_cast<size_t>(hf.H) * hf.W;
        if (npx == 0) continue;
        char* base = static_cast<char*>(dev_stage) + k * slot;
        float* d_pos = reinterpret_cast<float*>(base);
        float* d_nrm = reinterpret_cast<float*>(base + align_up(npx * 16, 256));
        float* d_sm = reinterpret_cast<float*>(base + 2 * align_up(npx * 16, 256));
        float* d_vis = reinterpret_cast<float*>(base + 2 * align_up(npx * 16, 256) +
                                                align_up(static_cast<size_t>(hf.Hs) * hf.Ws * 4, 256));
        if (i >= nslots) e = cudaStreamWaitEvent(cs, ctx->slot_d2h[k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pos, hf.pos4, npx * 16, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_nrm, hf.nrm4, npx * 16, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_sm, hf.sm, static_cast<size_t>(hf.Hs) * hf.Ws * 4, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->slot_h2d[k], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->slot_h2d[k], 0);
        if (e != cudaSuccess) break;
        nsm_frame df = hf;
        df.pos4 = d_pos;
        df.nrm4 = d_nrm;
        df.sm = d_sm;
        if ((s = nsm_infer(ctx, &df, w, precision, workspace, workspace_bytes, d_vis, stream)) != NSM_OK) {
            cudaStreamSynchronize(cs);
            cudaStreamSynchronize(ds);
            return s;
        }
        e = cudaEventRecord(ctx->slot_inf[k], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, ctx->slot_inf[k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vis_host[i], d_vis, npx * 4, cudaMemcpyDeviceToHost, ds);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->slot_d2h[k], ds);
    }
    const cudaError_t e1 = cudaStreamSynchronize(cs), e2 = cudaStreamSynchronize(ds), e3 = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "pipelined copies");
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "stream synchronize");
    return NSM_OK;
}

}  // extern "C"
