// Space-to-depth topology (Sec. 3.5): the two kernels around the tensor-core
// stages.
//   s2d_features  per half-resolution pixel (i, j): the gather of the four
//                 pixels (2i + a, 2j + b) of its 2x2 square, flattened into 16
//                 channels, channel 4 (2a + b) + c = feature c of offset (a, b),
//                 stored as BF16 hi + lo pairs [pixel][part][16] (the level-1
//                 encoder's input layout)
//   s2d_output    per full-resolution pixel: the bilinear x2 of head channel 0
//                 plus head channel 2a + b for square offsets (a, b) != (0, 0),
//                 then the sigmoid
#include <cuda_bf16.h>

#include "nsm_common.cuh"
#include "nsm_internal.h"

namespace nsm {

__global__ void __launch_bounds__(256) s2d_features_kernel(GatherParams g, uint16_t* __restrict__ out) {
    const int Hh = g.H / 2, Wh = g.W / 2;
    const size_t n = static_cast<size_t>(Hh) * Wh;
    for (size_t q = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; q < n;
         q += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(q / Wh), j = static_cast<int>(q % Wh);
        float f[16];
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const size_t p = static_cast<size_t>(2 * i + (ab >> 1)) * g.W + 2 * j + (ab & 1);
            const PixelGather o = gather_pixel(g, __ldg(g.pos4 + p), __ldg(g.nrm4 + p));
#pragma unroll
            for (int c = 0; c < 4; ++c) f[4 * ab + c] = o.f[c];
        }
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(f[2 * k]), h1 = __float2bfloat16_rn(f[2 * k + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(f[2 * k] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(f[2 * k + 1] - __bfloat162float(h1));
            hi[k] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
            lo[k] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + q * 32);
        dst[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        dst[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
        dst[2] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        dst[3] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
    }
}

__global__ void __launch_bounds__(256) s2d_output_kernel(const float4* __restrict__ o4, int H, int W,
                                                         float* __restrict__ vis) {
    const int Hh = H / 2, Wh = W / 2;
    const size_t n = static_cast<size_t>(H) * W;
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int y = static_cast<int>(p / W), x = static_cast<int>(p % W);
        const BilinTap ty = bilin_tap(y, Hh), tx = bilin_tap(x, Wh);
        const float c00 = __ldg(o4 + static_cast<size_t>(ty.i0) * Wh + tx.i0).x;
        const float c01 = __ldg(o4 + static_cast<size_t>(ty.i0) * Wh + tx.i1).x;
        const float c10 = __ldg(o4 + static_cast<size_t>(ty.i1) * Wh + tx.i0).x;
        const float c11 = __ldg(o4 + static_cast<size_t>(ty.i1) * Wh + tx.i1).x;
        float v = (c00 * tx.w0 + c01 * tx.w1) * ty.w0 + (c10 * tx.w0 + c11 * tx.w1) * ty.w1;
        const int ab = 2 * (y & 1) + (x & 1);
        if (ab) {
            const float4 d = __ldg(o4 + static_cast<size_t>(y >> 1) * Wh + (x >> 1));
            v += ab == 1 ? d.y : (ab == 2 ? d.z : d.w);
        }
        vis[p] = sigmoidf_acc(v);
    }
}

cudaError_t launch_s2d_features(const GatherParams& g, uint16_t* out, cudaStream_t stream) {
    const size_t n = static_cast<size_t>(g.H / 2) * (g.W / 2);
    if (n == 0) return cudaSuccess;
    const size_t cap = static_cast<size_t>(num_sms()) * 8;
    const size_t blocks = (n + 255) / 256;
    s2d_features_kernel<<<static_cast<unsigned>(blocks < cap ? blocks : cap), 256, 0, stream>>>(g, out);
    return cudaGetLastError();
}

cudaError_t launch_s2d_output(const float* o4, int H, int W, float* vis, cudaStream_t stream) {
    const size_t n = static_cast<size_t>(H) * W;
    if (n == 0) return cudaSuccess;
    const size_t cap = static_cast<size_t>(num_sms()) * 8;
    const size_t blocks = (n + 255) / 256;
    s2d_output_kernel<<<static_cast<unsigned>(blocks < cap ? blocks : cap), 256, 0, stream>>>(
        reinterpret_cast<const float4*>(o4), H, W, vis);
    return cudaGetLastError();
}

}  // namespace nsm
