// Shadow-map feature gather kernel (Sec. 3.1, 3.2): texel lookup, hard depth
// test, the four network inputs, and the optional blocker search with the
// penumbra-width model (Sec. 3.6, suppl. Sec. 4).
#include "nsm_common.cuh"
#include "nsm_internal.h"

namespace nsm {

constexpr int kMaxBlockerHalf = 32;

// Blocker search for one pixel: min / max of the texels z < z_f - beta z_f in
// the (2k+1)^2 window around (i, j), clipped to the map.  k is computed in
// binary32: k = min(32, ceil((r * (Ws / 2)) / (z_f * tan_half_fov))).
__device__ __forceinline__ int blocker_half(const GatherParams& g, float zf) {
    const float q = __fdiv_rn(__fmul_rn(g.radius, g.half_Ws), __fmul_rn(zf, g.tan_half_fov));
    const float kf = ceilf(q);
    return (kf <= static_cast<float>(kMaxBlockerHalf)) ? static_cast<int>(kf) : kMaxBlockerHalf;
}

// Penumbra width x_a + x_b of the spherical-occluder model (suppl. Sec. 4).
__device__ __forceinline__ float penumbra_width(float zf, float zmin, float zmax, float re) {
    const float zm = 0.5f * (zmax + zmin);
    const float rs = 0.5f * (zmax - zmin);
    const float td = asinf(rs / sqrtf(zm * zm + re * re));
    const float bq = re * (zf - zm) / zm;
    const float th = atanf((bq + re) / zf);
    return zf * tanf(th - td) - re + (zf * tanf(th + td) - re);
}

// One thread per pixel; full warps cover 32 consecutive pixels so the hard
// bits of a warp form one 32-bit word (ballot).
__global__ void __launch_bounds__(256) features_kernel(GatherParams g, float* __restrict__ feat,
                                                      int32_t* __restrict__ texel_out,
                                                      uint32_t* __restrict__ hard_out,
                                                      float* __restrict__ blocker_out) {
    const size_t npx = static_cast<size_t>(g.H) * g.W;
    const size_t nwords = (npx + 31) / 32;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t base = static_cast<size_t>(blockIdx.x) * blockDim.x; base < nwords * 32; base += stride) {
        const size_t p = base + threadIdx.x;
        const bool valid = p < npx;
        PixelGather o{};
        if (valid) {
            const float4 P = __ldg(g.pos4 + p);
            const float4 N = __ldg(g.nrm4 + p);
            o = gather_pixel(g, P, N);
            feat[p] = o.f[0];
            feat[npx + p] = o.f[1];
            feat[2 * npx + p] = o.f[2];
            feat[3 * npx + p] = o.f[3];
            if (texel_out) texel_out[p] = o.tex;
            if (blocker_out) {
                float zmin = 0.0f, zmax = 0.0f, width = 0.0f;
                if (o.tex >= 0) {
                    const int ci = o.tex % g.Ws, cj = o.tex / g.Ws;
                    const int k = blocker_half(g, o.zf);
                    const float thr = __fsub_rn(o.zf, __fmul_rn(g.beta, o.zf));
                    float lo = INFINITY, hi = -INFINITY;
                    const int j0 = max(0, cj - k), j1 = min(g.Hs - 1, cj + k);
                    const int i0 = max(0, ci - k), i1 = min(g.Ws - 1, ci + k);
                    for (int jj = j0; jj <= j1; ++jj) {
                        const float* row = g.sm + static_cast<size_t>(jj) * g.Ws;
                        for (int ii = i0; ii <= i1; ++ii) {
                            const float z = __ldg(row + ii);
                            if (z < thr) { lo = fminf(lo, z); hi = fmaxf(hi, z); }
                        }
                    }
                    if (lo <= hi) {
                        zmin = lo; zmax = hi;
                        width = penumbra_width(o.zf, zmin, zmax, g.radius);
                    }
                }
                blocker_out[p] = zmin;
                blocker_out[npx + p] = zmax;
                blocker_out[2 * npx + p] = width;
            }
        }
        if (hard_out) {
            const unsigned bits = __ballot_sync(0xffffffffu, valid && o.lit);
            if ((threadIdx.x & 31) == 0 && p < npx) hard_out[p >> 5] = bits;
        }
    }
}

cudaError_t launch_features(const GatherParams& g, float* feat, int32_t* texel_out, uint32_t* hard_out,
                            float* blocker_out, cudaStream_t stream) {
    const size_t npx = static_cast<size_t>(g.H) * g.W;
    if (npx == 0) return cudaSuccess;
    const int threads = 256;
    const size_t blocks_needed = (npx + threads - 1) / threads;
    int sms = num_sms();
    const size_t cap = static_cast<size_t>(sms) * 8;
    const int blocks = static_cast<int>(blocks_needed < cap ? blocks_needed : cap);
    features_kernel<<<blocks, threads, 0, stream>>>(g, feat, texel_out, hard_out, blocker_out);
    return cudaGetLastError();
}

}  // namespace nsm
