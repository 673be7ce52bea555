// Deeper networks for large penumbrae (Sec. 3.6): the encoder / decoder of
// Sec. 3.5 with L levels, L = 2 .. 7 (the paper's depth study uses 3, 5 and 7:
// receptive fields of 24, 96 and 384 pixels), FP32 on CUDA cores.  Channel
// plan as for three levels: widths w_l = 16 * 2^l; encoder level l: 3x3
// w_{l-1} -> w_l (4 features at level 0), 1x1 w_l -> w_l, average pooling;
// bottleneck: 3x3 w_{L-2} -> w_{L-1}, 1x1 w_{L-1} -> w_{L-2}; decoder level l:
// bilinear x2 of the coarser output plus the level's encoder output (l >= 1),
// 3x3 w_l -> w_l, 1x1 w_l -> w_{l-1} (16 at level 0); head 16 -> 1 and the
// sigmoid.  Levels 0 and 1 (the 3-level network's shapes) run as the training
// forward's fused kernels (encoder: 3x3, ReLU, 1x1, skip and pooling in one
// kernel; decoder: up-sampling while staging, 3x3, ReLU, 1x1); the coarser,
// wider levels run one kernel per layer on NHWC FP32 tensors in the
// workspace, the wide layers blocked over channels.
#include <vector>

#include "nsm_internal.h"
#include "train_internal.h"

namespace nsm {

struct DeepLayer {
    int cin, cout, k;
    size_t w, b;  // offsets in the canonical vector
};

static std::vector<DeepLayer> deep_layers(int L) {
    std::vector<DeepLayer> t;
    auto wd = [](int l) { return 16 << l; };
    size_t off = 0;
    auto add = [&](int ci, int co, int k) {
        t.push_back({ci, co, k, off, off + static_cast<size_t>(ci) * co * k * k});
        off += static_cast<size_t>(ci) * co * k * k + co;
    };
    for (int l = 0; l < L - 1; ++l) {
        add(l == 0 ? 4 : wd(l - 1), wd(l), 3);
        add(wd(l), wd(l), 1);
    }
    add(wd(L - 2), wd(L - 1), 3);
    add(wd(L - 1), wd(L - 2), 1);
    for (int l = L - 2; l >= 0; --l) {
        add(wd(l), wd(l), 3);
        add(wd(l), l >= 1 ? wd(l - 1) : 16, 1);
    }
    add(16, 1, 1);
    return t;
}

static size_t deep_param_count(int L) {
    const std::vector<DeepLayer> t = deep_layers(L);
    return t.back().b + 1;
}

// workspace: gather parameters, features (4), five full-resolution 16-channel
// FP32 tensors (every level's tensors fit: w_l (H W / 4^l) <= 16 H W), and the
// weights transposed to [tap][C_in][C_out] at their offsets in the vector
static size_t deep_ws_floats(int H, int W, int L) {
    return 64 + static_cast<size_t>(H) * W * (4 + 5 * 16) + deep_param_count(L);
}

}  // namespace nsm

using namespace nsm;

extern "C" {

size_t nsm_param_count_levels(int levels) {
    if (levels < 2 || levels > 7) return 0;
    return deep_param_count(levels);
}

size_t nsm_infer_deep_workspace_bytes(int H, int W, int levels) {
    if (H <= 0 || W <= 0 || levels < 2 || levels > 7) return 0;
    return deep_ws_floats(H, W, levels) * sizeof(float);
}

nsm_status nsm_infer_deep(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, int levels, void* workspace,
                          size_t workspace_bytes, float* vis_out, void* stream) {
    if (!ctx) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    if (levels < 2 || levels > 7) return fail(NSM_ERR_INVALID_ARG, "levels must be 2 .. 7, got %d", levels);
    nsm_status s = check_frame(frame, false);
    if (s != NSM_OK) return s;
    const int H = frame->H, W = frame->W;
    if (static_cast<size_t>(H) * W == 0) return NSM_OK;
    const int m = 1 << (levels - 1);
    if (H % m || W % m) return fail(NSM_ERR_SHAPE, "H, W must be multiples of 2^(levels - 1) = %d", m);
    if ((s = check_dev_ptr(dev_params, "dev_params", 4)) != NSM_OK || (s = check_dev_ptr(vis_out, "vis_out", 4)) != NSM_OK)
        return s;
    const size_t need = nsm_infer_deep_workspace_bytes(H, W, levels);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t hw = static_cast<size_t>(H) * W;
    float* base = static_cast<float*>(workspace);
    GatherParams* dgp = reinterpret_cast<GatherParams*>(base);
    static_assert(sizeof(GatherParams) <= 64 * sizeof(float), "gather parameters fit the workspace head");
    float* feat = base + 64;
    float* a3 = feat + 4 * hw;
    float* a1 = a3 + 16 * hw;
    float* h = a1 + 16 * hw;     // a level's input (pooled / bottleneck / decoder output)
    float* xin = h + 16 * hw;    // decoder input (up-sampled + skip)
    float* skip = xin + 16 * hw; // encoder outputs of levels 1 .. L-2, one after the other
    float* wt = base + 64 + hw * (4 + 5 * 16);  // transposed weights
    const GatherParams g = make_gather(frame);
    cudaError_t e = cudaMemcpyAsync(dgp, &g, sizeof(g), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = tr::features_batch(dgp, 1, H, W, feat, st);
    const std::vector<DeepLayer> Ls = deep_layers(levels);
    for (size_t i = 0; i + 1 < Ls.size() && e == cudaSuccess; ++i)  // every layer but the head
        e = tr::transpose_to_tap_major(dev_params + Ls[i].w, Ls[i].cin, Ls[i].cout, Ls[i].k, wt + Ls[i].w, st);
    auto wd = [](int l) { return 16 << l; };
    auto conv = [&](int li, const float* x, int relu_in, int Hl, int Wl, float* y) {
        const DeepLayer& d = Ls[li];
        return tr::conv_layer(d.cin, d.cout, d.k, x, relu_in, 1, Hl, Wl, wt + d.w, dev_params + d.b, y, st);
    };
    std::vector<float*> skips(levels, nullptr);
    const float* cur = feat;
    int li = 0;
    size_t skip_off = 0;
    // encoder: levels with the 3-level network's shapes (0, 1) in one fused
    // kernel each (3x3, ReLU, 1x1, skip, pooling); the pooled output never
    // overwrites the level's input
    for (int l = 0; l < levels - 1 && e == cudaSuccess; ++l, li += 2) {
        const int Hl = H >> l, Wl = W >> l;
        const DeepLayer &d3 = Ls[li], &d1 = Ls[li + 1];
        float* pooled = cur == h ? xin : h;
        if (l >= 1) {
            skips[l] = skip + skip_off;
            skip_off += static_cast<size_t>(Hl) * Wl * wd(l);
        }
        if (tr::enc_level_fusable(d3.cin, d3.cout)) {
            e = tr::enc_level_fused(d3.cin, d3.cout, cur, 1, Hl, Wl, wt + d3.w, dev_params + d3.b, dev_params + d1.w,
                                    dev_params + d1.b, skips[l], pooled, st);
        } else {
            e = conv(li, cur, 0, Hl, Wl, a3);
            if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, a1);
            if (e == cudaSuccess && l >= 1) e = tr::relu_copy(a1, static_cast<size_t>(Hl) * Wl * wd(l), skips[l], st);
            if (e == cudaSuccess) e = tr::pool_relu(a1, 1, Hl, Wl, wd(l), pooled, st);
        }
        cur = pooled;
    }
    const int Hb = H >> (levels - 1), Wb = W >> (levels - 1);
    if (e == cudaSuccess) e = conv(li++, cur, 0, Hb, Wb, a3);
    if (e == cudaSuccess) e = conv(li++, a3, 1, Hb, Wb, a1);
    if (e == cudaSuccess) e = tr::relu_copy(a1, static_cast<size_t>(Hb) * Wb * wd(levels - 2), h, st);
    // decoder: levels 1 and 0 up-sample while staging (fused kernels); a level
    // writes whichever scratch tensor its input does not occupy
    const float* lo = h;
    for (int l = levels - 2; l >= 0 && e == cudaSuccess; --l, li += 2) {
        const int Hl = H >> l, Wl = W >> l;
        const DeepLayer &d3 = Ls[li], &d1 = Ls[li + 1];
        if (tr::dec_level_fusable(d3.cin, d1.cout)) {
            // level 0 also applies the head (the layer after its 1x1) and writes only the visibility
            float* out = l >= 1 ? (lo == h ? a1 : h) : nullptr;
            e = tr::dec_level_fused(d3.cin, d1.cout, lo, l >= 1 ? skips[l] : nullptr, 1, Hl, Wl, wt + d3.w,
                                    dev_params + d3.b, dev_params + d1.w, dev_params + d1.b, l >= 1, out,
                                    l == 0 ? dev_params + Ls[li + 2].w : nullptr, l == 0 ? vis_out : nullptr, st);
            lo = out;
        } else {
            e = tr::up_add(lo, l >= 1 ? skips[l] : nullptr, 1, Hl, Wl, wd(l), xin, st);
            if (e == cudaSuccess) e = conv(li, xin, 0, Hl, Wl, a3);
            if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, a1);
            if (e == cudaSuccess && l >= 1) e = tr::relu_copy(a1, static_cast<size_t>(Hl) * Wl * wd(l - 1), h, st);
            lo = l >= 1 ? h : a1;
        }
    }
    if (e == cudaSuccess && lo) e = tr::head(lo, dev_params + Ls[li].w, hw, vis_out, st);
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "deep forward");
}

}  // extern "C"
