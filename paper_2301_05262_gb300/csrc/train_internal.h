// Internal declarations of the training path (train.cu).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "nsm_common.cuh"

namespace nsm {
namespace tr {

// FP32 NHWC buffers of one training / backward call, carved from one block:
// checkpoints for N views (features, level outputs, visibility) and the
// per-level recomputation scratch for the Nb views that are back-propagated.
struct Buffers {
    float *feat, *e0, *s1, *p1, *bo, *d1, *vis;
    float *gvis;
    float *xin, *a3, *a1, *ga1, *ga3, *gx, *glo, *gskip, *gtmp;
    float* wpart;  // per-CTA partial sums of the tensor-core weight gradients (kWgPartFloats)
};

// Floats of the partial-sum slots of one weight-gradient launch (8 MiB).
constexpr long long kWgPartFloats = 1ll << 21;

size_t workspace_floats(int N, int Nb, int H, int W);
Buffers carve(float* base, int N, int Nb, int H, int W);
cudaError_t features_batch(const GatherParams* dev_params, int N, int H, int W, float* feat, cudaStream_t st);
cudaError_t forward(const float* theta, const Buffers& b, int N, int Nb, int H, int W, cudaStream_t st);
cudaError_t backward(const float* theta, float* grad, const Buffers& b, int Nb, int H, int W, float* gfeat,
                     cudaStream_t st, const uint4* img = nullptr, int* err = nullptr);
// Tensor-core 3x3 convolutions of the backward (train_tc.cu): compensated
// BF16 operands (hi + lo pairs), FP32 accumulation, FP32 NHWC in and out.
// Images 2 l and 2 l + 1 are the l-th 3x3 layer (ENC0_3, ENC1_3, BOTT_3,
// DEC1_3, DEC0_3) and its data gradient (transposed, flipped weights), as
// 16-byte chunks at off[i] of one buffer of total_chunks chunks.
constexpr int kConv3Images = 10;
struct Conv3Images { int off[kConv3Images]; int total_chunks; };
Conv3Images conv3_images();
// Packs every image from the FP32 parameter vector (once per step).
cudaError_t conv3_pack(const float* theta, uint4* img, cudaStream_t st);
// y = conv3x3(x) (+ bias), zero padded; (cin, cout) one of the layers' shapes
// or their transposes (cudaErrorInvalidValue otherwise); err: device error
// word, set to 7 when a bounded wait gave up.  c1 > 0 (the level's 1x1 after
// the 3x3, (cin, cout, c1) one of the network's levels): also y1 = b1 + W1
// relu(y) (W1 OIHW [c1][cout]), in the separate 1x1 layer's summation order.
cudaError_t conv3_tc(int cin, int cout, const float* x, int N, int H, int W, const uint4* img, const float* bias,
                     float* y, int* err, cudaStream_t st, const float* w1 = nullptr, const float* b1 = nullptr,
                     int c1 = 0, float* y1 = nullptr);
// Tensor-core weight gradients (train_wgrad.cu): dW += sum_p g~[p][o] x~[p + tap][c]
// (OIHW), db += sum_p g~[p][o], x~ = relu(x) if relu_in, g~ = g (m > 0) if gm;
// k = 3 (zero padded) or 1.  Compensated BF16 operands, FP32 accumulation in
// tensor memory, per-CTA partial sums in part (kWgPartFloats floats) added in a
// fixed order: no atomics.  (cin, cout, k) one of the network's layers
// (cudaErrorInvalidValue otherwise); err: device error word, set to 8 when a
// bounded wait gave up.
cudaError_t wgrad_tc(int cin, int cout, int k, const float* x, int relu_in, const float* g, const float* gm, int N,
                     int H, int W, float* part, float* dW, float* db, int* err, cudaStream_t st);
// 1x1 weight gradients on CUDA cores (train_wgrad.cu): dW += sum_p g~[p][o]
// x~[p][c] (OIHW), db += sum_p g~[p][o], with x~ and g~ as for wgrad_tc; per-CTA
// partial sums in part added in a fixed order.  (cin, cout) one of the
// network's 1x1 layers (cudaErrorInvalidValue otherwise).
cudaError_t wgrad1x1_tiles(int cin, int cout, const float* x, int relu_in, const float* g, const float* gm, int N,
                           int H, int W, float* part, float* dW, float* db, cudaStream_t st);
// dW[e] += sum_s part[s][e] for e < nw, db[e - nw] += ... for nw <= e < entries, s in order.
cudaError_t slot_reduce(const float* part, int slots, int entries, int nw, float* dW, float* db, cudaStream_t st);
cudaError_t loss_l1(const float* vis, const float* target, int B, int T, size_t npx, float alpha, float* gvis,
                    float* loss, cudaStream_t st);
cudaError_t adam(float* theta, const float* grad, float* m, float* v, size_t n, float lr, float b1, float b2,
                 float eps, int step, cudaStream_t st);

// Forward layers of the deeper networks (FP32 NHWC; conv_layer: zero-padded
// "same" k x k convolution of relu?(x) plus bias, weights in the [tap][C_in]
// [C_out] layout transpose_to_tap_major writes from OIHW (16-byte aligned),
// cudaErrorInvalidValue for a shape outside the 2- to 7-level layer tables).
cudaError_t transpose_to_tap_major(const float* w, int cin, int cout, int k, float* wt, cudaStream_t st);
cudaError_t conv_layer(int cin, int cout, int k, const float* x, int relu_in, int N, int H, int W, const float* wt,
                       const float* b, float* y, cudaStream_t st);
bool enc_level_fusable(int cin, int cout);
bool dec_level_fusable(int cin, int cout1);
cudaError_t enc_level_fused(int cin, int cout, const float* x, int N, int H, int W, const float* wt3, const float* b3,
                            const float* w1, const float* b1, float* skip, float* pooled, cudaStream_t st);
cudaError_t dec_level_fused(int cin, int cout1, const float* lo, const float* skip, int N, int H, int W,
                            const float* wt3, const float* b3, const float* w1, const float* b1, int relu_out, float* y,
                            const float* wh, float* vis, cudaStream_t st);
// Tensor-core layers of the deeper networks' inner levels (deep_tc.cu):
// y = relu?(conv_k(relu?(x)) + b) (relu_out), FP32 NHWC [H][W][C], k = 3 (zero padded) or 1,
// compensated BF16 operands, FP32 accumulation.  Supported: C_in a multiple of
// 16 (k = 3) or 64 (k = 1), C_out a multiple of 32.  The weight image (packed
// from OIHW once per call, deep_tc_image_bytes bytes, 16-byte aligned) feeds
// deep_tc_conv; err: device error word, set to 9 when a bounded wait gave up.
bool deep_tc_supported(int cin, int cout, int k);
size_t deep_tc_image_bytes(int cin, int cout, int k);
cudaError_t deep_tc_pack(const float* w, int cin, int cout, int k, uint4* img, cudaStream_t st);
cudaError_t deep_tc_conv(int cin, int cout, int k, const float* x, int relu_in, int H, int W, const uint4* img,
                         const float* bias, float* y, int relu_out, int* err, cudaStream_t st);
// Three-term FP8 (E4M3) layers (fp8x3.cu): y = relu?(conv_k(relu?(x)) + b) on FP32
// NHWC tensors, k = 3 or 1, activations and per-output-channel-scaled weights
// as three E4M3 terms each (scales 1, 2^-4, 2^-8), products on tcgen05
// kind::f8f6f4 with FP32 accumulation.  Supported: C_in a multiple of 4, C_out a
// multiple of 16.  f8x3_pack writes the layer's image (f8x3_image_bytes bytes,
// 256-byte aligned: E4M3 weight terms, then the scales); err: device error
// word, set to 10 when a bounded wait gave up.
bool f8x3_supported(int cin, int cout, int k);
size_t f8x3_image_bytes(int cin, int cout, int k);
cudaError_t f8x3_pack(const float* w, int cin, int cout, int k, void* img, cudaStream_t st);
cudaError_t f8x3_conv(int cin, int cout, int k, const float* x, int relu_in, int H, int W, const void* img,
                      const float* bias, float* y, int relu_out, int* err, cudaStream_t st);
cudaError_t pool_relu(const float* x, int N, int H, int W, int C, float* y, cudaStream_t st);        // avg2x2(relu(x))
cudaError_t up_add(const float* lo, const float* skip, int N, int H, int W, int C, float* y, cudaStream_t st);
cudaError_t relu_copy(const float* x, size_t n, float* y, cudaStream_t st);
cudaError_t head(const float* a1, const float* wh, size_t npx, float* vis, cudaStream_t st);         // 16 -> 1, sigmoid

}  // namespace tr
}  // namespace nsm
