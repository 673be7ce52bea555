// E4M3 weight images of the FP8 tensor-core form (net_fp8.cu), built on the
// device from the canonical FP32 vector.  Every output channel o of a layer
// gets the scale s_o = max |W[o, ...]| / 448 (1 for an all-zero channel) and
// its weights are stored as e4m3(W / s_o) (round to nearest even, saturating);
// the stage kernels multiply the FP32 accumulator by s_o.
//
// Image layouts (16-byte chunks of 16 E4M3 weights; a K = 32 MMA step reads
// two chunks 3 * C_out chunks apart for the 3x3 forms, C_out apart for 1x1):
//   first level (C_in = 4):  chunk (h, ky, n): h = 0 holds [W[n][c][ky][kx]
//                            for kx = 0..2, c = 0..3 | 4 zero bytes], h = 1 zeros
//   3x3, C_in = 16:          chunk ((p, h), ky, n) = W[n][0..15][ky][2p + h]
//                            (zeros for kx = 3)
//   3x3, C_in = 32:          chunk ((kx, g), ky, n) = W[n][16g .. 16g+15][ky][kx]
//   1x1:                     chunk (g, n) = W[n][16g .. 16g+15], padded with a
//                            zero chunk row to an even count of groups
#include <cuda_fp8.h>

#include "nsm_internal.h"

namespace nsm {

F8Images fp8_images() {
    F8Images im{};
    size_t pos = 0, spos = 0;
    for (int l = 0; l < HEAD; ++l) {
        const LayerShape& s = kLayers[l];
        size_t chunks;
        if (s.k == 3) chunks = static_cast<size_t>(s.cin == 4 ? 6 : (s.cin == 16 ? 12 : 18)) * s.cout;
        else chunks = static_cast<size_t>((s.cin / 16 + 1) / 2 * 2) * s.cout;
        im.img_off[l] = pos;
        im.scale_off[l] = spos;
        pos += chunks * 16;
        spos += s.cout;
    }
    im.img_bytes = pos;
    im.scales = spos;
    return im;
}

__device__ __forceinline__ uint8_t to_e4m3(float v) {
    return static_cast<uint8_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
}

struct LayerTab { LayerShape l[NUM_LAYERS]; };

// one thread per (layer, output channel)
__global__ void pack_fp8_kernel(const float* __restrict__ params, uint8_t* __restrict__ img,
                                float* __restrict__ scales, F8Images im, LayerOffsets off, LayerTab tab) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int l = 0;
    for (; l < HEAD; ++l) {
        if (t < tab.l[l].cout) break;
        t -= tab.l[l].cout;
    }
    if (l >= HEAD) return;
    const LayerShape s = tab.l[l];
    const int n = t, taps = s.k * s.k;
    const float* W = params + off.w[l] + static_cast<size_t>(n) * s.cin * taps;  // W[n][c][tap]
    float mx = 0.f;
    for (int i = 0; i < s.cin * taps; ++i) mx = fmaxf(mx, fabsf(W[i]));
    const float sc = mx > 0.f ? mx / 448.f : 1.f;
    scales[im.scale_off[l] + n] = sc;
    uint8_t* base = img + im.img_off[l];
    auto wq = [&](int c, int tap) { return to_e4m3(W[c * taps + tap] / sc); };
    auto chunk = [&](size_t idx) { return base + idx * 16; };
    const size_t C = s.cout;
    if (s.k == 3 && s.cin == 4) {
        for (int h = 0; h < 2; ++h)
            for (int ky = 0; ky < 3; ++ky) {
                uint8_t* q = chunk((static_cast<size_t>(h) * 3 + ky) * C + n);
                for (int e = 0; e < 16; ++e) {
                    const int kx = e / 4, c = e % 4;
                    q[e] = (h == 0 && kx < 3) ? wq(c, ky * 3 + kx) : 0;
                }
            }
    } else if (s.k == 3 && s.cin == 16) {
        for (int kx4 = 0; kx4 < 4; ++kx4)
            for (int ky = 0; ky < 3; ++ky) {
                uint8_t* q = chunk((static_cast<size_t>(kx4) * 3 + ky) * C + n);
                for (int e = 0; e < 16; ++e) q[e] = kx4 < 3 ? wq(e, ky * 3 + kx4) : 0;
            }
    } else if (s.k == 3) {  // C_in = 32
        for (int kx = 0; kx < 3; ++kx)
            for (int g = 0; g < 2; ++g)
                for (int ky = 0; ky < 3; ++ky) {
                    uint8_t* q = chunk(((static_cast<size_t>(kx) * 2 + g) * 3 + ky) * C + n);
                    for (int e = 0; e < 16; ++e) q[e] = wq(16 * g + e, ky * 3 + kx);
                }
    } else {
        const int mp = s.cin / 16, mpp = (mp + 1) / 2 * 2;
        for (int g = 0; g < mpp; ++g) {
            uint8_t* q = chunk(static_cast<size_t>(g) * C + n);
            for (int e = 0; e < 16; ++e) q[e] = g < mp ? wq(16 * g + e, 0) : 0;
        }
    }
}

cudaError_t launch_pack_fp8(const float* params, uint8_t* img, float* scales, cudaStream_t stream) {
    int total = 0;
    for (int l = 0; l < HEAD; ++l) total += kLayers[l].cout;
    LayerTab tab;
    for (int l = 0; l < NUM_LAYERS; ++l) tab.l[l] = kLayers[l];
    pack_fp8_kernel<<<(total + 127) / 128, 128, 0, stream>>>(params, img, scales, fp8_images(), layer_offsets(), tab);
    return cudaGetLastError();
}

}  // namespace nsm
