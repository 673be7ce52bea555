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
//
// Tensor-core form (nsm_infer_deep_ex with NSM_BF16): levels 0 and 1 have the
// 3-level network's shapes, so they run on its compensated-BF16 stage kernels
// (gather + level-0 encoder, level-1 encoder with skip, level-1 decoder,
// level-0 decoder on the coarse grid with the head), their weight images
// packed from this network's vector; the inner levels 2 .. L-1 run one
// tcgen05 layer per 3x3 / 1x1 (deep_tc.cu) on FP32 NHWC tensors, entering
// from the level-1 encoder's pooled BF16 pairs and leaving as the FP32
// input the level-1 decoder up-samples.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "ctx_internal.h"
#include "nsm_internal.h"
#include "tc_stage.h"
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

// Layers of the inner levels (2 .. L-1): indices [4, 4L - 6) of deep_layers;
// the 3-level network's layers map to 0 .. 3 (encoders), 4L - 6 .. 4L - 3
// (decoders) and 4L - 2 (head).
static int deep_index_of(Layer l, int L) {
    switch (l) {
        case ENC0_3: return 0; case ENC0_1: return 1; case ENC1_3: return 2; case ENC1_1: return 3;
        case DEC1_3: return 4 * L - 6; case DEC1_1: return 4 * L - 5;
        case DEC0_3: return 4 * L - 4; case DEC0_1: return 4 * L - 3;
        case HEAD: return 4 * L - 2;
        default: return -1;
    }
}

// Packed weights of one form, laid out from one 256-byte-aligned base (a
// workspace region or a nsm_deep_weights allocation): FP32, every layer's
// weights as [tap][C_in][C_out] at its canonical offset; BF16, the stage
// kernels' images of levels 0 and 1 (the 3-level packing table with this
// network's offsets), the table, then the inner levels' tcgen05 images;
// FP8, every layer's three-term E4M3 image.  The head stays in the FP32
// vector.
struct DeepImgs {
    const float* wt = nullptr;
    const uint16_t* img16 = nullptr;
    std::vector<const void*> layer;
};

static size_t deep_images_bytes(int L, nsm_precision p) {
    const std::vector<DeepLayer> t = deep_layers(L);
    if (p == NSM_FP32) return align_up(deep_param_count(L) * sizeof(float), 256);
    size_t b = 0;
    if (p == NSM_BF16) {
        b += align_up(bf16_images().total * sizeof(uint16_t), 256) + align_up(pack_desc_bytes() * NUM_LAYERS, 256);
        for (int i = 4; i < 4 * L - 6; ++i) b += align_up(tr::deep_tc_image_bytes(t[i].cin, t[i].cout, t[i].k), 256);
    } else {
        for (size_t i = 0; i + 1 < t.size(); ++i) b += align_up(tr::f8x3_image_bytes(t[i].cin, t[i].cout, t[i].k), 256);
    }
    return b;
}

// BF16 hi + lo pairs [n][2][C] -> FP32 [n][C] (another buffer)
template <int C>
__global__ void deep_pairs_to_f32_kernel(const uint16_t* __restrict__ in, size_t n, float* __restrict__ out) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n * C;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const size_t p = i / C, c = i % C;
        out[i] = __bfloat162float(__ushort_as_bfloat16(in[p * 2 * C + c])) +
                 __bfloat162float(__ushort_as_bfloat16(in[p * 2 * C + C + c]));
    }
}

// The L-level network with every convolution in the three-term FP8 form (packed
// weights P), one layer per kernel on FP32 NHWC tensors (features, a3, a1, h,
// xin, skip: the FP32 form's workspace regions), as the FP32 form's unfused
// levels run.
static cudaError_t deep_forward_f8x3(nsm_ctx* ctx, const nsm_frame* frame, const float* params, int L,
                                     const DeepImgs& P, GatherParams* dgp, float* feat, float* a3, float* a1, float* h,
                                     float* xin, float* skip, float* vis, cudaStream_t st) {
    const int H = frame->H, W = frame->W;
    const std::vector<DeepLayer> Ls = deep_layers(L);
    const std::vector<const void*>& img = P.layer;
    cudaError_t e = cudaSuccess;
    const GatherParams g = make_gather(frame);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dgp, &g, sizeof(g), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = tr::features_batch(dgp, 1, H, W, feat, st);
    auto wd = [](int l) { return 16 << l; };
    auto conv = [&](int li, const float* x, int relu_in, int Hl, int Wl, float* y, int relu_out = 0) {
        const DeepLayer& d = Ls[li];
        return tr::f8x3_conv(d.cin, d.cout, d.k, x, relu_in, Hl, Wl, img[li], params + d.b, y, relu_out, ctx->d_err,
                             st);
    };
    std::vector<float*> skips(L, nullptr);
    const float* cur = feat;
    size_t skip_off = 0;
    int li = 0;
    for (int l = 0; l < L - 1 && e == cudaSuccess; ++l, li += 2) {
        const int Hl = H >> l, Wl = W >> l;
        float* pooled = cur == h ? xin : h;
        // the 1x1 writes its rectified output: the skip (levels >= 1) or a1; the pooling reads it
        float* out1 = a1;
        if (l >= 1) {
            skips[l] = skip + skip_off;
            skip_off += static_cast<size_t>(Hl) * Wl * wd(l);
            out1 = skips[l];
        }
        e = conv(li, cur, 0, Hl, Wl, a3);
        if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, out1, 1);
        if (e == cudaSuccess) e = tr::pool_relu(out1, 1, Hl, Wl, wd(l), pooled, st);
        cur = pooled;
    }
    const int Hb = H >> (L - 1), Wb = W >> (L - 1);
    if (e == cudaSuccess) e = conv(li++, cur, 0, Hb, Wb, a3);
    if (e == cudaSuccess) e = conv(li++, a3, 1, Hb, Wb, h, 1);  // cur was read by the 3x3 already
    const float* lo = h;
    for (int l = L - 2; l >= 0 && e == cudaSuccess; --l, li += 2) {
        const int Hl = H >> l, Wl = W >> l;
        e = tr::up_add(lo, l >= 1 ? skips[l] : nullptr, 1, Hl, Wl, wd(l), xin, st);
        if (e == cudaSuccess) e = conv(li, xin, 0, Hl, Wl, a3);
        // levels >= 1: the rectified output into h (read by the up-sampling already); level 0: a1 for the head
        if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, l >= 1 ? h : a1, l >= 1 ? 1 : 0);
        lo = l >= 1 ? h : a1;
    }
    if (e == cudaSuccess) e = tr::head(lo, params + Ls[li].w, static_cast<size_t>(H) * W, vis, st);
    return e;
}

// Pack the form's weights from the device vector into base (deep_images_bytes).
static cudaError_t deep_pack(const float* params, int L, nsm_precision p, char* base, DeepImgs* out, cudaStream_t st) {
    const std::vector<DeepLayer> Ls = deep_layers(L);
    *out = DeepImgs{};
    out->layer.assign(Ls.size(), nullptr);
    cudaError_t e = cudaSuccess;
    if (p == NSM_FP32) {
        float* wt = reinterpret_cast<float*>(base);
        out->wt = wt;
        for (size_t i = 0; i + 1 < Ls.size() && e == cudaSuccess; ++i)  // every layer but the head
            e = tr::transpose_to_tap_major(params + Ls[i].w, Ls[i].cin, Ls[i].cout, Ls[i].k, wt + Ls[i].w, st);
        return e;
    }
    char* q = base;
    if (p == NSM_FP8) {
        for (size_t i = 0; i + 1 < Ls.size() && e == cudaSuccess; ++i) {
            out->layer[i] = q;
            e = tr::f8x3_pack(params + Ls[i].w, Ls[i].cin, Ls[i].cout, Ls[i].k, q, st);
            q += align_up(tr::f8x3_image_bytes(Ls[i].cin, Ls[i].cout, Ls[i].k), 256);
        }
        return e;
    }
    const BF16Images im = bf16_images();
    uint16_t* img16 = reinterpret_cast<uint16_t*>(q);
    out->img16 = img16;
    q += align_up(im.total * sizeof(uint16_t), 256);
    void* ddesc = q;
    q += align_up(pack_desc_bytes() * NUM_LAYERS, 256);
    // the stage kernels' weight images, packed from this network's levels 0 and 1
    PackDescHost desc[NUM_LAYERS];
    int nd = 0;
    for (int i = 0; i < im.n; ++i) {
        int layer = -1;
        for (int l = 0; l < NUM_LAYERS; ++l)
            if (im.desc[i].img_off == im.img_off[l] && kLayers[l].cin == im.desc[i].cin) layer = l;
        const int di = layer < 0 ? -1 : deep_index_of(static_cast<Layer>(layer), L);
        if (di < 0) continue;  // the 3-level bottleneck: replaced by the inner levels
        desc[nd] = im.desc[i];
        desc[nd].w_off = Ls[di].w;
        ++nd;
    }
    e = cudaMemcpyAsync(ddesc, desc, pack_desc_bytes() * nd, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_pack_bf16(params, img16, ddesc, nd, st);
    for (int i = 4; i < 4 * L - 6 && e == cudaSuccess; ++i) {
        out->layer[i] = q;
        e = tr::deep_tc_pack(params + Ls[i].w, Ls[i].cin, Ls[i].cout, Ls[i].k, reinterpret_cast<uint4*>(q), st);
        q += align_up(tr::deep_tc_image_bytes(Ls[i].cin, Ls[i].cout, Ls[i].k), 256);
    }
    return e;
}

// The L-level network with levels 0, 1 on the BF16 stage kernels and the inner
// levels on the tcgen05 layers, from packed weights P; a3, a1, h, xin, skip:
// the FP32 form's workspace regions (16 H W floats each), actb: the stage
// kernels' activations (activations_bytes).
static cudaError_t deep_forward_bf16(nsm_ctx* ctx, const nsm_frame* frame, const float* params, int L,
                                     const DeepImgs& P, float* a3, float* a1, float* h, float* xin, float* skip,
                                     char* actb, float* vis, cudaStream_t st) {
    const int H = frame->H, W = frame->W;
    const std::vector<DeepLayer> Ls = deep_layers(L);
    Activations act{};
    activations_bytes(H, W, 4, &act, actb);
    const BF16Images im = bf16_images();
    const uint16_t* img16 = P.img16;
    const std::vector<const void*>& mid = P.layer;
    cudaError_t e = cudaSuccess;
    auto I = [&](Layer l) { return reinterpret_cast<const uint4*>(img16 + im.img_off[l]); };
    const GatherParams g = make_gather(frame);
    const int head = deep_index_of(HEAD, L);
    auto stage = [&](int s, Layer l3, Layer l1) {
        TcBatch b{};
        b.nviews = 1;
        b.b3img = I(l3);
        b.b1img = I(l1);
        const DeepLayer &d3 = Ls[deep_index_of(l3, L)], &d1 = Ls[deep_index_of(l1, L)];
        b.bias3 = params + d3.b;
        b.bias1 = params + d1.b;
        b.w3 = params + d3.w;
        b.w1 = params + d1.w;
        b.head = params + Ls[head].w;  // head weights followed by its bias
        b.err = ctx->d_err;
        TcJob& j = b.job[0];
        j.g = g;
        switch (s) {
            case 0: j.H = H; j.W = W; j.out = static_cast<uint16_t*>(act.e0); break;
            case 1: j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(act.e0);
                    j.out_skip = static_cast<float*>(act.s1); j.out = static_cast<uint16_t*>(act.p1); break;
            case 3: j.H = H / 2; j.W = W / 2; j.in_f = static_cast<const float*>(act.bo);
                    j.skip = static_cast<const float*>(act.s1); j.out = static_cast<uint16_t*>(act.d1); break;
            default: j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(act.d1); j.vis = vis; break;
        }
        return tc_launch_stage(s, tc_default_variant(s), b, 0, st);
    };
    if ((e = stage(0, ENC0_3, ENC0_1)) != cudaSuccess || (e = stage(1, ENC1_3, ENC1_1)) != cudaSuccess) return e;
    // inner levels on FP32 NHWC tensors, from the pooled level-1 output
    auto wd = [](int l) { return 16 << l; };
    auto conv = [&](int li, const float* x, int relu_in, int Hl, int Wl, float* y, int relu_out = 0) {
        const DeepLayer& d = Ls[li];
        return tr::deep_tc_conv(d.cin, d.cout, d.k, x, relu_in, Hl, Wl, static_cast<const uint4*>(mid[li]),
                                params + d.b, y, relu_out, ctx->d_err, st);
    };
    const size_t n2 = static_cast<size_t>(H / 4) * (W / 4);
    deep_pairs_to_f32_kernel<32><<<static_cast<int>(std::min<size_t>((n2 * 32 + 255) / 256, 4096)), 256, 0, st>>>(
        static_cast<const uint16_t*>(act.p1), n2, xin);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const float* cur = xin;
    std::vector<float*> skips(L, nullptr);
    size_t skip_off = 0;
    int li = 4;
    for (int l = 2; l < L - 1 && e == cudaSuccess; ++l, li += 2) {
        const int Hl = H >> l, Wl = W >> l;
        float* pooled = cur == h ? xin : h;
        skips[l] = skip + skip_off;
        skip_off += static_cast<size_t>(Hl) * Wl * wd(l);
        // the 1x1 writes the rectified skip directly; the pooling reads it
        e = conv(li, cur, 0, Hl, Wl, a3);
        if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, skips[l], 1);
        if (e == cudaSuccess) e = tr::pool_relu(skips[l], 1, Hl, Wl, wd(l), pooled, st);
        cur = pooled;
    }
    const int Hb = H >> (L - 1), Wb = W >> (L - 1);
    if (e == cudaSuccess) e = conv(li++, cur, 0, Hb, Wb, a3);
    if (e == cudaSuccess) e = conv(li++, a3, 1, Hb, Wb, h, 1);  // cur was read by the 3x3 already
    for (int l = L - 2; l >= 2 && e == cudaSuccess; --l, li += 2) {
        const int Hl = H >> l, Wl = W >> l;
        e = tr::up_add(h, skips[l], 1, Hl, Wl, wd(l), xin, st);
        if (e == cudaSuccess) e = conv(li, xin, 0, Hl, Wl, a3);
        if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, h, 1);  // h was read by the up-sampling
    }
    if (e != cudaSuccess) return e;
    // the level-2 output (32 channels at H / 4) is what the level-1 decoder up-samples
    act.bo = h;
    if ((e = stage(3, DEC1_3, DEC1_1)) != cudaSuccess) return e;
    return stage(4, DEC0_3, DEC0_1);
}

// The FP32 form from packed weights P (P.wt): levels 0 and 1 as the training
// forward's fused kernels, the coarser levels one kernel per layer.
static cudaError_t deep_forward_fp32(const nsm_frame* frame, const float* params, int levels, const DeepImgs& P,
                                     GatherParams* dgp, float* feat, float* a3, float* a1, float* h, float* xin,
                                     float* skip, float* vis_out, cudaStream_t st) {
    const int H = frame->H, W = frame->W;
    const size_t hw = static_cast<size_t>(H) * W;
    const float* wt = P.wt;
    const GatherParams g = make_gather(frame);
    cudaError_t e = cudaMemcpyAsync(dgp, &g, sizeof(g), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = tr::features_batch(dgp, 1, H, W, feat, st);
    const std::vector<DeepLayer> Ls = deep_layers(levels);
    auto wd = [](int l) { return 16 << l; };
    auto conv = [&](int li, const float* x, int relu_in, int Hl, int Wl, float* y) {
        const DeepLayer& d = Ls[li];
        return tr::conv_layer(d.cin, d.cout, d.k, x, relu_in, 1, Hl, Wl, wt + d.w, params + d.b, y, st);
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
            e = tr::enc_level_fused(d3.cin, d3.cout, cur, 1, Hl, Wl, wt + d3.w, params + d3.b, params + d1.w,
                                    params + d1.b, skips[l], pooled, st);
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
                                    params + d3.b, params + d1.w, params + d1.b, l >= 1, out,
                                    l == 0 ? params + Ls[li + 2].w : nullptr, l == 0 ? vis_out : nullptr, st);
            lo = out;
        } else {
            e = tr::up_add(lo, l >= 1 ? skips[l] : nullptr, 1, Hl, Wl, wd(l), xin, st);
            if (e == cudaSuccess) e = conv(li, xin, 0, Hl, Wl, a3);
            if (e == cudaSuccess) e = conv(li + 1, a3, 1, Hl, Wl, a1);
            if (e == cudaSuccess && l >= 1) e = tr::relu_copy(a1, static_cast<size_t>(Hl) * Wl * wd(l - 1), h, st);
            lo = l >= 1 ? h : a1;
        }
    }
    if (e == cudaSuccess && lo) e = tr::head(lo, params + Ls[li].w, hw, vis_out, st);
    return e;
}

// Workspace of one call: the gather parameters, the features and five
// 16 H W-float scratch tensors (every level's tensors fit: w_l (H W / 4^l) <= 16
// H W), then for the BF16 form the stage kernels' activations.
static size_t deep_region_bytes(int H, int W) {
    return align_up((64 + static_cast<size_t>(H) * W * (4 + 5 * 16)) * sizeof(float), 256);
}
static size_t deep_act_bytes(int H, int W, nsm_precision p) {
    return p == NSM_BF16 ? activations_bytes(H, W, 4, nullptr, nullptr) : 0;
}

// One forward from packed weights P, the workspace laid out as above.
static cudaError_t deep_run(nsm_ctx* ctx, const nsm_frame* frame, const float* params, int levels, nsm_precision p,
                            const DeepImgs& P, void* workspace, float* vis_out, cudaStream_t st) {
    const size_t hw = static_cast<size_t>(frame->H) * frame->W;
    float* base = static_cast<float*>(workspace);
    GatherParams* dgp = reinterpret_cast<GatherParams*>(base);
    static_assert(sizeof(GatherParams) <= 64 * sizeof(float), "gather parameters fit the workspace head");
    float* feat = base + 64;
    float* a3 = feat + 4 * hw;
    float* a1 = a3 + 16 * hw;
    float* h = a1 + 16 * hw;     // a level's input (pooled / bottleneck / decoder output)
    float* xin = h + 16 * hw;    // decoder input (up-sampled + skip)
    float* skip = xin + 16 * hw; // encoder outputs of levels 1 .. L-2, one after the other
    char* actb = static_cast<char*>(workspace) + deep_region_bytes(frame->H, frame->W);
    if (p == NSM_FP8)
        return deep_forward_f8x3(ctx, frame, params, levels, P, dgp, feat, a3, a1, h, xin, skip, vis_out, st);
    if (p == NSM_BF16) return deep_forward_bf16(ctx, frame, params, levels, P, a3, a1, h, xin, skip, actb, vis_out, st);
    return deep_forward_fp32(frame, params, levels, P, dgp, feat, a3, a1, h, xin, skip, vis_out, st);
}

// Shared checks of the deep entry points (frame, levels, form).
static nsm_status deep_check(nsm_ctx* ctx, const nsm_frame* frame, int levels, nsm_precision precision) {
    if (!ctx) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    if (levels < 2 || levels > 7) return fail(NSM_ERR_INVALID_ARG, "levels must be 2 .. 7, got %d", levels);
    if (precision != NSM_FP32 && precision != NSM_BF16 && precision != NSM_FP8)
        return fail(NSM_ERR_UNSUPPORTED, "the deeper networks run in the FP32, BF16 or three-term FP8 form");
    if (precision == NSM_BF16 && levels < 3)
        return fail(NSM_ERR_UNSUPPORTED, "the BF16 form needs 3 or more levels, got %d", levels);
    nsm_status s = check_frame(frame, false);
    if (s != NSM_OK) return s;
    const int m = 1 << (levels - 1);
    if (frame->H % m || frame->W % m) return fail(NSM_ERR_SHAPE, "H, W must be multiples of 2^(levels - 1) = %d", m);
    return NSM_OK;
}

}  // namespace nsm

// Packed weights of an L-level network in one form (nsm_deep_weights_create).
struct nsm_deep_weights {
    int device;
    int levels;
    nsm_precision precision;
    size_t n;
    float* d_params;   // canonical FP32 vector (biases and the head are read from it)
    char* d_images;    // deep_images_bytes of the form
    nsm::DeepImgs imgs;
};

using namespace nsm;

extern "C" {

size_t nsm_param_count_levels(int levels) {
    if (levels < 2 || levels > 7) return 0;
    return deep_param_count(levels);
}

size_t nsm_infer_deep_workspace_bytes(int H, int W, int levels) {
    return nsm_infer_deep_ex_workspace_bytes(H, W, levels, NSM_FP32);
}

size_t nsm_infer_deep_ex_workspace_bytes(int H, int W, int levels, nsm_precision precision) {
    if (H <= 0 || W <= 0 || levels < 2 || levels > 7) return 0;
    if (precision != NSM_FP32 && precision != NSM_BF16 && precision != NSM_FP8) return 0;
    if (precision == NSM_BF16 && levels < 3) return 0;
    return deep_region_bytes(H, W) + deep_act_bytes(H, W, precision) + deep_images_bytes(levels, precision);
}

nsm_status nsm_infer_deep(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, int levels, void* workspace,
                          size_t workspace_bytes, float* vis_out, void* stream) {
    return nsm_infer_deep_ex(ctx, frame, dev_params, levels, NSM_FP32, workspace, workspace_bytes, vis_out, stream);
}

nsm_status nsm_infer_deep_ex(nsm_ctx* ctx, const nsm_frame* frame, const float* dev_params, int levels,
                             nsm_precision precision, void* workspace, size_t workspace_bytes, float* vis_out,
                             void* stream) {
    nsm_status s = deep_check(ctx, frame, levels, precision);
    if (s != NSM_OK) return s;
    const int H = frame->H, W = frame->W;
    if (static_cast<size_t>(H) * W == 0) return NSM_OK;
    if ((s = check_dev_ptr(dev_params, "dev_params", 4)) != NSM_OK || (s = check_dev_ptr(vis_out, "vis_out", 4)) != NSM_OK)
        return s;
    const size_t need = nsm_infer_deep_ex_workspace_bytes(H, W, levels, precision);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the weights packed per call after the call's own regions
    char* images = static_cast<char*>(workspace) + deep_region_bytes(H, W) + deep_act_bytes(H, W, precision);
    DeepImgs P;
    cudaError_t e = deep_pack(dev_params, levels, precision, images, &P, st);
    if (e == cudaSuccess) e = deep_run(ctx, frame, dev_params, levels, precision, P, workspace, vis_out, st);
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "deep forward");
}

nsm_status nsm_deep_weights_create(nsm_ctx* ctx, const float* host_params, size_t n, int levels,
                                   nsm_precision precision, nsm_deep_weights** out) {
    if (!ctx || !host_params || !out) return fail(NSM_ERR_INVALID_ARG, "ctx, host_params and out must be non-NULL");
    *out = nullptr;
    if (levels < 2 || levels > 7) return fail(NSM_ERR_INVALID_ARG, "levels must be 2 .. 7, got %d", levels);
    if (precision != NSM_FP32 && precision != NSM_BF16 && precision != NSM_FP8)
        return fail(NSM_ERR_UNSUPPORTED, "the deeper networks run in the FP32, BF16 or three-term FP8 form");
    if (precision == NSM_BF16 && levels < 3)
        return fail(NSM_ERR_UNSUPPORTED, "the BF16 form needs 3 or more levels, got %d", levels);
    if (n != deep_param_count(levels))
        return fail(NSM_ERR_SHAPE, "parameter vector has %zu floats, expected %zu", n, deep_param_count(levels));
    if (n > static_cast<size_t>(INT32_MAX) || !finite_all(host_params, static_cast<int>(n)))
        return fail(NSM_ERR_INVALID_ARG, "parameters must be finite");
    nsm_deep_weights* w = new nsm_deep_weights{};
    cudaGetDevice(&w->device);
    w->levels = levels;
    w->precision = precision;
    w->n = n;
    cudaError_t e = cudaMalloc(&w->d_params, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w->d_images, deep_images_bytes(levels, precision));
    if (e == cudaSuccess) e = cudaMemcpy(w->d_params, host_params, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = deep_pack(w->d_params, levels, precision, w->d_images, &w->imgs, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        nsm_deep_weights_destroy(w);
        return cuda_fail(e, "deep weights");
    }
    *out = w;
    return NSM_OK;
}

nsm_status nsm_deep_weights_load_device(nsm_deep_weights* w, const float* dev_params, size_t n, void* stream) {
    if (!w) return fail(NSM_ERR_INVALID_ARG, "weights are NULL");
    if (n != w->n) return fail(NSM_ERR_SHAPE, "%zu floats given, the weights hold %zu", n, w->n);
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != w->device) return fail(NSM_ERR_INVALID_ARG, "weights live on device %d, current device %d", w->device, dev);
    nsm_status s = check_dev_ptr(dev_params, "dev_params", 4);
    if (s != NSM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(w->d_params, dev_params, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = deep_pack(w->d_params, w->levels, w->precision, w->d_images, &w->imgs, st);
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "deep weights repack");
}

void nsm_deep_weights_destroy(nsm_deep_weights* w) {
    if (!w) return;
    cudaFree(w->d_params);
    cudaFree(w->d_images);
    delete w;
}

size_t nsm_infer_deep_packed_workspace_bytes(int H, int W, int levels, nsm_precision precision) {
    if (nsm_infer_deep_ex_workspace_bytes(H, W, levels, precision) == 0) return 0;
    return deep_region_bytes(H, W) + deep_act_bytes(H, W, precision);
}

nsm_status nsm_infer_deep_packed(nsm_ctx* ctx, const nsm_frame* frame, const nsm_deep_weights* w, void* workspace,
                                 size_t workspace_bytes, float* vis_out, void* stream) {
    if (!w) return fail(NSM_ERR_INVALID_ARG, "weights are NULL");
    nsm_status s = deep_check(ctx, frame, w->levels, w->precision);
    if (s != NSM_OK) return s;
    const int H = frame->H, W = frame->W;
    if (static_cast<size_t>(H) * W == 0) return NSM_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != w->device) return fail(NSM_ERR_INVALID_ARG, "weights live on device %d, current device %d", w->device, dev);
    if ((s = check_dev_ptr(vis_out, "vis_out", 4)) != NSM_OK) return s;
    const size_t need = nsm_infer_deep_packed_workspace_bytes(H, W, w->levels, w->precision);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    const cudaError_t e = deep_run(ctx, frame, w->d_params, w->levels, w->precision, w->imgs, workspace, vis_out,
                                   static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "deep forward (packed weights)");
}

}  // extern "C"
