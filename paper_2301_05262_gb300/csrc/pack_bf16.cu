// Packing of the network weights into the tensor-core operand images
// (shared-memory layout of each layer's B operand, BF16 hi + lo parts).
#include <cuda_bf16.h>

#include "nsm_internal.h"

namespace nsm {

// ------------------------------------------------------------------ weight packing
// Shared-memory images of the BF16 weights, each weight w stored as
// hi = bf16(w) and lo = bf16(w - hi), stacked along the output rows of every
// K block (rows 0 .. c_out-1 hi, rows c_out .. 2 c_out-1 lo), so one MMA of
// width 2 c_out multiplies by both (16-byte chunks of 8 K values):
//   3x3, C_in >= 16:  chunk (tap, g, n) = W[n][8g .. 8g+7][tap]
//   3x3 first level:  chunk (k, h, n)   = tap t = 2k + h (t < 9), channels
//                     [c0..c3 | c0..c3] (the same weight for the hi and lo
//                     parts of each feature), zero for t = 9
//   1x1:              chunk (g, n)      = W[n][8g .. 8g+7]
// Row-stacked 3x3 forms (the three kernel rows ky stacked along the output
// rows as well, so one MMA over an input row feeds three output rows):
//   3x3, C_in >= 16:  chunk (kx, g, ky, n) = W[n][8g .. 8g+7][ky][kx]
//   3x3 first level:  chunk (p, h, ky, n)  = column kx = 2p + h (zero for
//                     kx = 3), channels [c0..c3 | c0..c3] as above
// Coarse-grid form of an up-sampling decoder level (bilinear x2 then 3x3):
//   chunk (tap, g, n), n = 16 p + o for output parity p = 2a + b:
//   E[p][o][8g .. 8g+7][tap], where the effective weight of coarse offset
//   (dy, dx) = tap is  E = sum_{ky,kx} W[o][c][ky][kx] q(a, ky, dy) q(b, kx, dx)
//   and q(a, k, d) is the bilinear weight of coarse index i + d - 1 in fine
//   index 2i + a + k - 1 (1/4 or 3/4, half-pixel centres), summed in FP64.
using PackDesc = PackDescHost;

__device__ double up_coef(int a, int k, int d) {
    const int t = a + k - 1;           // fine index 2i + t
    const int m = t >= 0 ? t / 2 : -1;  // = floor(t / 2)
    const int par = t - 2 * m;
    const int off = d - 1;
    if (par == 0) return off == m - 1 ? 0.25 : (off == m ? 0.75 : 0.0);
    return off == m ? 0.75 : (off == m + 1 ? 0.25 : 0.0);
}

__global__ void pack_bf16_kernel(const float* __restrict__ params, uint16_t* __restrict__ img,
                                 const PackDesc* __restrict__ descs, int ndesc) {
    for (int d = 0; d < ndesc; ++d) {
        const PackDesc pd = descs[d];
        for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < pd.count;
             i += static_cast<size_t>(gridDim.x) * blockDim.x) {
            const int e = static_cast<int>(i % 8);
            const size_t chunk = i / 8;
            float v = 0.f;
            if (pd.kind == 0) {  // 3x3 general: chunk = (tap * (cin/8) + g) * cout + n
                const int n = static_cast<int>(chunk % pd.cout);
                const size_t t2 = chunk / pd.cout;
                const int g = static_cast<int>(t2 % (pd.cin / 8));
                const int tap = static_cast<int>(t2 / (pd.cin / 8));
                v = params[pd.w_off + (static_cast<size_t>(n) * pd.cin + 8 * g + e) * 9 + tap];
            } else if (pd.kind == 1) {  // first level hi/lo: chunk = (k * 2 + h) * cout + n
                const int n = static_cast<int>(chunk % pd.cout);
                const int kh = static_cast<int>(chunk / pd.cout);
                const int tap = kh;  // = 2k + h
                if (tap < 9) v = params[pd.w_off + (static_cast<size_t>(n) * 4 + (e % 4)) * 9 + tap];
            } else if (pd.kind == 3) {  // stacked 3x3: chunk = ((kx * (cin/8) + g) * 3 + ky) * cout + n
                const int n = static_cast<int>(chunk % pd.cout);
                const size_t t2 = chunk / pd.cout;
                const int ky = static_cast<int>(t2 % 3);
                const size_t t3 = t2 / 3;
                const int g = static_cast<int>(t3 % (pd.cin / 8));
                const int kx = static_cast<int>(t3 / (pd.cin / 8));
                v = params[pd.w_off + (static_cast<size_t>(n) * pd.cin + 8 * g + e) * 9 + ky * 3 + kx];
            } else if (pd.kind == 4) {  // stacked first level: chunk = ((p * 2 + h) * 3 + ky) * cout + n
                const int n = static_cast<int>(chunk % pd.cout);
                const size_t t2 = chunk / pd.cout;
                const int ky = static_cast<int>(t2 % 3);
                const int kx = static_cast<int>(t2 / 3);  // = 2p + h
                if (kx < 3) v = params[pd.w_off + (static_cast<size_t>(n) * 4 + (e % 4)) * 9 + ky * 3 + kx];
            } else if (pd.kind == 5) {  // coarse-grid 3x3: chunk = (tap * (cin/8) + g) * cout + n
                const int n = static_cast<int>(chunk % pd.cout);
                const size_t t2 = chunk / pd.cout;
                const int g = static_cast<int>(t2 % (pd.cin / 8));
                const int tap = static_cast<int>(t2 / (pd.cin / 8));
                const int co = pd.cout / 4, p = n / co, o = n % co, a = p >> 1, b = p & 1;
                const int dy = tap / 3, dx = tap % 3;
                double acc = 0.0;
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        const double q = up_coef(a, ky, dy) * up_coef(b, kx, dx);
                        if (q != 0.0)
                            acc += q * params[pd.w_off + (static_cast<size_t>(o) * pd.cin + 8 * g + e) * 9 + ky * 3 + kx];
                    }
                v = static_cast<float>(acc);
            } else {  // 1x1: chunk = g * cout + n
                const int n = static_cast<int>(chunk % pd.cout);
                const int g = static_cast<int>(chunk / pd.cout);
                v = params[pd.w_off + static_cast<size_t>(n) * pd.cin + 8 * g + e];
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            // hi and lo weights stacked along the output rows of each K block:
            // rows [0, cout) hold the hi parts, rows [cout, 2 cout) the lo parts
            const size_t blk = chunk / pd.cout, n = chunk % pd.cout;
            const size_t base = blk * 2 * pd.cout;
            img[pd.img_off + (base + n) * 8 + e] = __bfloat16_as_ushort(hi);
            img[pd.img_off + (base + pd.cout + n) * 8 + e] = __bfloat16_as_ushort(lo);
        }
    }
}

BF16Images bf16_images(bool s2d) {
    const LayerOffsets off = s2d ? layer_offsets_s2d() : layer_offsets();
    BF16Images im{};
    size_t pos = 0;
    auto add = [&](int layer, int kind) {
        const int ci = kLayers[layer].cin, co = (kind == 5 ? 4 : 1) * kLayers[layer].cout;
        size_t count;
        if (kind == 0 || kind == 3 || kind == 5) count = static_cast<size_t>(9) * ci * co;
        else if (kind == 1) count = static_cast<size_t>(10) * co * 8;
        else if (kind == 4) count = static_cast<size_t>(12) * co * 8;
        else count = static_cast<size_t>(ci) * co;
        im.desc[im.n] = {kind, ci, co, off.w[layer], pos, count};
        im.img_off[layer] = pos;
        pos += 2 * count;  // hi and lo parts (counts are multiples of 8)
        ++im.n;
    };
    // a 3x3 layer is row-stacked when its three stacked kernel rows (3 x 2 c_out
    // MMA rows) fit one MMA of width <= 256
    auto k3 = [&](int layer) { return 3 * 2 * kLayers[layer].cout <= 256 ? 3 : 0; };
    if (!s2d) { add(ENC0_3, 3 * 2 * kLayers[ENC0_3].cout <= 256 ? 4 : 1); add(ENC0_1, 2); }
    add(ENC1_3, k3(ENC1_3)); add(ENC1_1, 2); add(BOTT_3, k3(BOTT_3)); add(BOTT_1, 2);
    add(DEC1_3, k3(DEC1_3)); add(DEC1_1, 2);
    // the level-0 decoder runs on the coarse grid: effective weights of its 4 output parities
    if (!s2d) { add(DEC0_3, 5); add(DEC0_1, 2); }
    im.total = pos;
    return im;
}

cudaError_t launch_pack_bf16(const float* params, uint16_t* img, const void* dev_descs, int ndesc, cudaStream_t stream) {
    pack_bf16_kernel<<<64, 256, 0, stream>>>(params, img, static_cast<const PackDesc*>(dev_descs), ndesc);
    return cudaGetLastError();
}

size_t pack_desc_bytes() { return sizeof(PackDesc); }

}  // namespace nsm
