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
                                                      uint32_t* __restrict__ hard_out) {
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
        }
        if (hard_out) {
            const unsigned bits = __ballot_sync(0xffffffffu, valid && o.lit);
            if ((threadIdx.x & 31) == 0 && p < npx) hard_out[p >> 5] = bits;
        }
    }
}


// ------------------------------------------------------------------ blocker search
// Two kernels.  blocker_table_kernel writes, once per map, the min and max of
// every 8 x 8 and every 4 x 4 square of texels (T8 / T4 [y][x] over the
// squares whose top-left texel is (x, y), clipped at the map's edges; float2
// (min, max), row stride Ws): ~4x the map's bytes, read back from L2.  Then
// blocker_kernel takes one thread per pixel (16 x 16 pixel CTAs, so a CTA's
// windows overlap in L1).  A window is covered by rows of 8 x 8 squares (the
// last row / column overlaps the previous one; at most 9 x 9 squares for the
// 65-texel windows), a row's entries loaded together.  Per square the window
// minimum takes its min; a square whose max is below the pixel's threshold
// contributes its max (all its texels are blockers); one whose min is below
// the threshold and max is not is split into its four 4 x 4 squares, tested
// the same way, and a 4 x 4 square that straddles the threshold has its 16
// texels scanned.  Windows narrower than 8 texels are scanned directly.
// Min / max are order independent and every texel of a window is covered, so
// results equal the exhaustive scan exactly.
constexpr int kBTile = 16;                 // pixels per CTA side (256 threads)
constexpr int kTabX = 64, kTabY = 16;      // table entries per CTA of blocker_table_kernel

// T8 / T4 [y][x] = (min, max) of the 8 x 8 / 4 x 4 texels from (x, y), clipped
// at the map's edges (row stride Ws)
__global__ void __launch_bounds__(256) blocker_table_kernel(const float* __restrict__ sm, int Ws, int Hs,
                                                            float2* __restrict__ T8, float2* __restrict__ T4) {
    __shared__ float sZ[kTabY + 7][kTabX + 8];
    __shared__ float sMn4[kTabY + 7][kTabX], sMx4[kTabY + 7][kTabX];
    __shared__ float sMn8[kTabY + 7][kTabX], sMx8[kTabY + 7][kTabX];
    const int x0 = blockIdx.x * kTabX, y0 = blockIdx.y * kTabY, tid = threadIdx.x;
    // clamping the coordinates clips the squares at the edges (repeated texels
    // do not change a min or max)
    for (int idx = tid; idx < (kTabY + 7) * (kTabX + 7); idx += blockDim.x) {
        const int yy = idx / (kTabX + 7), xx = idx % (kTabX + 7);
        sZ[yy][xx] = __ldg(sm + static_cast<size_t>(min(y0 + yy, Hs - 1)) * Ws + min(x0 + xx, Ws - 1));
    }
    __syncthreads();
    for (int idx = tid; idx < (kTabY + 7) * kTabX; idx += blockDim.x) {
        const int yy = idx / kTabX, xx = idx % kTabX;
        float a = sZ[yy][xx], b = a, c, d;
#pragma unroll
        for (int e = 1; e < 4; ++e) { a = fminf(a, sZ[yy][xx + e]); b = fmaxf(b, sZ[yy][xx + e]); }
        c = a; d = b;
#pragma unroll
        for (int e = 4; e < 8; ++e) { c = fminf(c, sZ[yy][xx + e]); d = fmaxf(d, sZ[yy][xx + e]); }
        sMn4[yy][xx] = a; sMx4[yy][xx] = b;
        sMn8[yy][xx] = c; sMx8[yy][xx] = d;
    }
    __syncthreads();
    for (int idx = tid; idx < kTabY * kTabX; idx += blockDim.x) {
        const int yy = idx / kTabX, xx = idx % kTabX;
        if (y0 + yy >= Hs || x0 + xx >= Ws) continue;
        float a = sMn4[yy][xx], b = sMx4[yy][xx], c = sMn8[yy][xx], d = sMx8[yy][xx];
#pragma unroll
        for (int e = 1; e < 4; ++e) { a = fminf(a, sMn4[yy + e][xx]); b = fmaxf(b, sMx4[yy + e][xx]); }
#pragma unroll
        for (int e = 1; e < 8; ++e) { c = fminf(c, sMn8[yy + e][xx]); d = fmaxf(d, sMx8[yy + e][xx]); }
        const size_t o = static_cast<size_t>(y0 + yy) * Ws + x0 + xx;
        T4[o] = make_float2(a, b);
        T8[o] = make_float2(c, d);
    }
}

__global__ void __launch_bounds__(kBTile * kBTile) blocker_kernel(GatherParams g, const float2* __restrict__ T8,
                                                                  const float2* __restrict__ T4,
                                                                  float* __restrict__ blocker_out) {
    const int tid = threadIdx.x;
    const int lx = tid % kBTile, ly = tid / kBTile;
    const int tx = blockIdx.x * kBTile + lx, ty = blockIdx.y * kBTile + ly;
    if (tx >= g.W || ty >= g.H) return;
    const size_t npx = static_cast<size_t>(g.H) * g.W;
    const size_t p = static_cast<size_t>(ty) * g.W + tx;
    const float4 P = __ldg(g.pos4 + p);
    int ci = 0, cj = 0;
    float zmin = 0.0f, zmax = 0.0f, width = 0.0f;
    if (texel_index(g, P.x, P.y, P.z, &ci, &cj) >= 0) {
        const float zf = emitter_distance(g, P.x, P.y, P.z);
        const float thr = __fsub_rn(zf, __fmul_rn(g.beta, zf));
        const int k = blocker_half(g, zf);
        const int i0 = max(0, ci - k), i1 = min(g.Ws - 1, ci + k);
        const int j0 = max(0, cj - k), j1 = min(g.Hs - 1, cj + k);
        const int wx = i1 - i0 + 1, wy = j1 - j0 + 1;
        float lo = INFINITY, hi = -INFINITY;
        if (wx >= 8 && wy >= 8) {
            const int nx = (wx + 7) >> 3;  // squares per row, <= 9
            for (int yq = 0;; yq += 8) {
                const int ys = min(yq, wy - 8) + j0;
                const float2* trow = T8 + static_cast<size_t>(ys) * g.Ws + i0;
                float2 t[9];
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    t[q] = q < nx ? __ldg(trow + min(8 * q, wx - 8)) : make_float2(INFINITY, -INFINITY);
                unsigned straddle = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    lo = fminf(lo, t[q].x);
                    if (t[q].y < thr) hi = fmaxf(hi, t[q].y);
                    else if (t[q].x < thr) straddle |= 1u << q;
                }
                while (straddle) {
                    const int q = __ffs(straddle) - 1;
                    straddle &= straddle - 1;
                    const size_t o = static_cast<size_t>(ys) * g.Ws + min(8 * q, wx - 8) + i0;
                    float2 u[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) u[h] = __ldg(T4 + o + (h >> 1) * 4 * static_cast<size_t>(g.Ws) + (h & 1) * 4);
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        if (u[h].y < thr) {
                            hi = fmaxf(hi, u[h].y);
                        } else if (u[h].x < thr) {
                            const float* r0 = g.sm + o + (h >> 1) * 4 * static_cast<size_t>(g.Ws) + (h & 1) * 4;
                            float z[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e) z[e] = __ldg(r0 + static_cast<size_t>(e >> 2) * g.Ws + (e & 3));
#pragma unroll
                            for (int e = 0; e < 16; ++e) if (z[e] < thr) hi = fmaxf(hi, z[e]);
                        }
                    }
                }
                if (yq + 8 >= wy) break;
            }
        } else {
            for (int yy = j0; yy <= j1; ++yy)
                for (int xx = i0; xx <= i1; ++xx) {
                    const float z = __ldg(g.sm + static_cast<size_t>(yy) * g.Ws + xx);
                    lo = fminf(lo, z);
                    if (z < thr) hi = fmaxf(hi, z);
                }
        }
        if (lo < thr) {
            zmin = lo;
            zmax = hi;
            width = penumbra_width(zf, zmin, zmax, g.radius);
        }
    }
    blocker_out[p] = zmin;
    blocker_out[npx + p] = zmax;
    blocker_out[2 * npx + p] = width;
}

cudaError_t launch_features(const GatherParams& g, float* feat, int32_t* texel_out, uint32_t* hard_out,
                            float* blocker_out, void* table_ws, cudaStream_t stream) {
    const size_t npx = static_cast<size_t>(g.H) * g.W;
    if (npx == 0) return cudaSuccess;
    const int threads = 256;
    const size_t blocks_needed = (npx + threads - 1) / threads;
    int sms = num_sms();
    const size_t cap = static_cast<size_t>(sms) * 8;
    const int blocks = static_cast<int>(blocks_needed < cap ? blocks_needed : cap);
    features_kernel<<<blocks, threads, 0, stream>>>(g, feat, texel_out, hard_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !blocker_out) return e;
    // the tables: the caller's workspace, else stream-ordered scratch from the library's pool
    void* tab = table_ws;
    const size_t nt = static_cast<size_t>(g.Ws) * g.Hs;
    if (!tab) {
        cudaMemPool_t pool;
        if ((e = scratch_pool(&pool)) != cudaSuccess) return e;
        e = cudaMallocFromPoolAsync(&tab, 2 * nt * sizeof(float2), pool, stream);
        if (e != cudaSuccess) return e;
    }
    float2* t8 = static_cast<float2*>(tab);
    float2* t4 = t8 + nt;
    const dim3 tgrid((g.Ws + kTabX - 1) / kTabX, (g.Hs + kTabY - 1) / kTabY);
    blocker_table_kernel<<<tgrid, 256, 0, stream>>>(g.sm, g.Ws, g.Hs, t8, t4);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const dim3 grid((g.W + kBTile - 1) / kBTile, (g.H + kBTile - 1) / kBTile);
        blocker_kernel<<<grid, kBTile * kBTile, 0, stream>>>(g, t8, t4, blocker_out);
        e = cudaGetLastError();
    }
    const cudaError_t ef = table_ws ? cudaSuccess : cudaFreeAsync(tab, stream);
    return e != cudaSuccess ? e : ef;
}

}  // namespace nsm
