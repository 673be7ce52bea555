// Shadow-map feature gather kernel (Sec. 3.1, 3.2): texel lookup, hard depth
// test, the four network inputs, and the optional blocker search with the
// penumbra-width model (Sec. 3.6, suppl. Sec. 4).
#include <climits>

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
// One CTA per 16 x 16 pixel tile (one thread per pixel).  The union of a
// pixel group's search windows (bounding box from warp-level min / max
// reductions of the window corners, then across warps) is staged in shared
// memory and reduced to the min and max of every 8 x 8 square of the box (a
// row pass over all outputs, then a column pass in place, band by band).  A
// pixel's window is covered by 8 x 8 squares (the last row / column of
// squares overlaps the previous one); per square the window minimum takes its
// min; a square whose max is below the pixel's threshold contributes its max
// (all its texels are blockers); one whose min is below the threshold and max
// is not has its 64 texels scanned.  Windows narrower than 8 texels are
// scanned directly.  Pixel groups: the whole tile when its box fits the
// staging arrays, else each 8 x 8 quadrant in turn; a pixel whose quadrant box
// does not fit either is scanned in global memory by its whole warp (coalesced
// row loads, shuffle reductions).  Min / max are order independent and every
// texel of a window is covered, so results equal the exhaustive scan exactly.
constexpr int kBTile = 16;                 // pixels per tile side (256 threads)
constexpr int kBoxCap = 9216;              // staged texels per array (three arrays)
constexpr int kBlockerSmem = 3 * kBoxCap * 4;

struct BlkPixel {
    int i0, i1, j0, j1;   // clipped window (empty: i0 > i1)
    float thr;
};

// stage the box [bx0, bx0 + BW) x [by0, by0 + BH) and build the 8 x 8 min / max tables
__device__ __forceinline__ void blk_stage(const GatherParams& g, int bx0, int by0, int BW, int BH, float* sZ,
                                          float* sMn, float* sMx) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint32_t z0 = static_cast<uint32_t>(__cvta_generic_to_shared(sZ));
    if ((bx0 & 3) == 0 && (BW & 3) == 0 && (g.Ws & 3) == 0) {
        // 16-byte async copies (box aligned to 4 texels by the caller when the map allows)
        const int bw4 = BW / 4;
        for (int idx = tid; idx < bw4 * BH; idx += nt) {
            const int yy = idx / bw4, xx = 4 * (idx % bw4);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(z0 + 4u * (yy * BW + xx)),
                         "l"(g.sm + static_cast<size_t>(by0 + yy) * g.Ws + bx0 + xx) : "memory");
        }
    } else {
        for (int idx = tid; idx < BW * BH; idx += nt) {  // 4-byte async copies, all in flight
            const int yy = idx / BW, xx = idx % BW;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(z0 + 4u * idx),
                         "l"(g.sm + static_cast<size_t>(by0 + yy) * g.Ws + bx0 + xx) : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // rows: sMn / sMx[y][x] = min / max of sZ[y][x .. x+7]
    for (int idx = tid; idx < BW * BH; idx += nt) {
        const int xx = idx % BW;
        if (xx + 7 < BW) {
            float a = sZ[idx], b = a;
#pragma unroll
            for (int d = 1; d < 8; ++d) { a = fminf(a, sZ[idx + d]); b = fmaxf(b, sZ[idx + d]); }
            sMn[idx] = a;
            sMx[idx] = b;
        }
    }
    __syncthreads();
    // columns, in place in bands of 8 rows: a band's outputs read rows up to
    // 7 below it, which later bands have not overwritten yet
    // band height: at most 5 outputs per thread (BW <= kBoxCap / 8 = 1152 when BH >= 8)
    const int hb = max(1, min(8, 5 * nt / BW));
    for (int y0 = 0; y0 + 7 < BH; y0 += hb) {
        const int rows = min(hb, BH - 7 - y0);
        const int n = rows * BW;
        float a[5], b[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int idx = tid + q * nt;
            a[q] = b[q] = 0.f;
            if (idx < n && idx % BW + 7 < BW) {
                const int base = (y0 + idx / BW) * BW + idx % BW;
                a[q] = sMn[base];
                b[q] = sMx[base];
#pragma unroll
                for (int d = 1; d < 8; ++d) {
                    a[q] = fminf(a[q], sMn[base + d * BW]);
                    b[q] = fmaxf(b[q], sMx[base + d * BW]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int idx = tid + q * nt;
            if (idx < n && idx % BW + 7 < BW) {
                const int base = (y0 + idx / BW) * BW + idx % BW;
                sMn[base] = a[q];
                sMx[base] = b[q];
            }
        }
        __syncthreads();
    }
}

// one pixel's query against a staged box
__device__ __forceinline__ void blk_query(const BlkPixel& px, int bx0, int by0, int BW, const float* sZ,
                                          const float* sMn, const float* sMx, float& lo, float& hi) {
    const int wx = px.i1 - px.i0 + 1, wy = px.j1 - px.j0 + 1;
    const int x0 = px.i0 - bx0, y0 = px.j0 - by0;
    const float thr = px.thr;
    if (wx >= 8 && wy >= 8) {
        for (int yq = 0;; yq += 8) {
            const int ys = min(yq, wy - 8) + y0;
            for (int xq = 0;; xq += 8) {
                const int xs = min(xq, wx - 8) + x0;
                const float smn = sMn[ys * BW + xs], smx = sMx[ys * BW + xs];
                lo = fminf(lo, smn);
                if (smx < thr) {
                    hi = fmaxf(hi, smx);
                } else if (smn < thr) {
                    for (int dy = 0; dy < 8; ++dy) {
                        const float* r = sZ + (ys + dy) * BW + xs;
#pragma unroll
                        for (int dx = 0; dx < 8; ++dx) if (r[dx] < thr) hi = fmaxf(hi, r[dx]);
                    }
                }
                if (xq + 8 >= wx) break;
            }
            if (yq + 8 >= wy) break;
        }
    } else {
        for (int yy = y0; yy < y0 + wy; ++yy)
            for (int xx = x0; xx < x0 + wx; ++xx) {
                const float z = sZ[yy * BW + xx];
                lo = fminf(lo, z);
                if (z < thr) hi = fmaxf(hi, z);
            }
    }
}

// bounding box of the windows of the threads with `in` set: warp reductions, then across warps
__device__ __forceinline__ void blk_box(const BlkPixel& px, bool in, int (*sBox)[kBTile * kBTile / 32], int& bx0,
                                        int& bx1, int& by0, int& by1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool use = in && px.i0 <= px.i1;
    int b0 = use ? px.i0 : INT_MAX, b1 = use ? px.i1 : INT_MIN, b2 = use ? px.j0 : INT_MAX, b3 = use ? px.j1 : INT_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b0 = min(b0, __shfl_xor_sync(0xffffffffu, b0, o));
        b1 = max(b1, __shfl_xor_sync(0xffffffffu, b1, o));
        b2 = min(b2, __shfl_xor_sync(0xffffffffu, b2, o));
        b3 = max(b3, __shfl_xor_sync(0xffffffffu, b3, o));
    }
    __syncthreads();  // sBox free
    if (lane == 0) { sBox[0][warp] = b0; sBox[1][warp] = b1; sBox[2][warp] = b2; sBox[3][warp] = b3; }
    __syncthreads();
    bx0 = INT_MAX; bx1 = INT_MIN; by0 = INT_MAX; by1 = INT_MIN;
#pragma unroll
    for (int w = 0; w < kBTile * kBTile / 32; ++w) {
        bx0 = min(bx0, sBox[0][w]); bx1 = max(bx1, sBox[1][w]);
        by0 = min(by0, sBox[2][w]); by1 = max(by1, sBox[3][w]);
    }
}

__global__ void __launch_bounds__(kBTile * kBTile) blocker_kernel(GatherParams g, float* __restrict__ blocker_out) {
    extern __shared__ __align__(16) float bsm[];
    float* sZ = bsm;
    float* sMn = bsm + kBoxCap;
    float* sMx = bsm + 2 * kBoxCap;
    __shared__ int sBox[4][kBTile * kBTile / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    const int lx = tid % kBTile, ly = tid / kBTile;
    const int tx = blockIdx.x * kBTile + lx, ty = blockIdx.y * kBTile + ly;
    const bool valid = tx < g.W && ty < g.H;
    const size_t npx = static_cast<size_t>(g.H) * g.W;
    const size_t p = valid ? static_cast<size_t>(ty) * g.W + tx : 0;
    BlkPixel px{1, 0, 1, 0, 0.f};
    float zf = 0.f;
    bool act = false;
    if (valid) {
        const float4 P = __ldg(g.pos4 + p);
        int ci = 0, cj = 0;
        if (texel_index(g, P.x, P.y, P.z, &ci, &cj) >= 0) {
            act = true;
            zf = emitter_distance(g, P.x, P.y, P.z);
            px.thr = __fsub_rn(zf, __fmul_rn(g.beta, zf));
            const int k = blocker_half(g, zf);
            px.i0 = max(0, ci - k); px.i1 = min(g.Ws - 1, ci + k);
            px.j0 = max(0, cj - k); px.j1 = min(g.Hs - 1, cj + k);
        }
    }
    float lo = INFINITY, hi = -INFINITY;
    bool done = !act;
    // the whole tile, else its four quadrants in turn
    for (int grp = 0; grp < 5; ++grp) {
        const bool mine = grp == 0 || (grp - 1) == ((ly >= 8) * 2 + (lx >= 8));
        int bx0, bx1, by0, by1;
        blk_box(px, mine && !done, sBox, bx0, bx1, by0, by1);
        if (bx0 > bx1) {
            if (grp == 0) break;  // nothing left in the tile
            continue;
        }
        if ((g.Ws & 3) == 0) {  // widen the box to 16-byte boundaries of the map rows
            bx0 &= ~3;
            bx1 |= 3;
        }
        const int BW = bx1 - bx0 + 1, BH = by1 - by0 + 1;
        if (static_cast<long long>(BW) * BH > kBoxCap) continue;
        blk_stage(g, bx0, by0, BW, BH, sZ, sMn, sMx);
        if (mine && !done) {
            blk_query(px, bx0, by0, BW, sZ, sMn, sMx, lo, hi);
            done = true;
        }
        __syncthreads();  // staging arrays reused by the next group
        if (grp == 0) break;
    }
    // what is left: one warp per pixel over the map in global memory
    unsigned left = __ballot_sync(0xffffffffu, !done);
    while (left) {
        const int src = __ffs(left) - 1;
        left &= left - 1;
        const int i0 = __shfl_sync(0xffffffffu, px.i0, src), i1 = __shfl_sync(0xffffffffu, px.i1, src);
        const int j0 = __shfl_sync(0xffffffffu, px.j0, src), j1 = __shfl_sync(0xffffffffu, px.j1, src);
        const float thr = __shfl_sync(0xffffffffu, px.thr, src);
        float a = INFINITY, b = -INFINITY;
        // up to 3 columns per lane (windows are at most 65 wide), 8 rows of loads in flight
        for (int jb = j0; jb <= j1; jb += 8) {
            float z[8][3];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int jj = jb + r, ii = i0 + lane + 32 * c;
                    z[r][c] = (jj <= j1 && ii <= i1) ? __ldg(g.sm + static_cast<size_t>(jj) * g.Ws + ii) : INFINITY;
                }
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a = fminf(a, z[r][c]);
                    if (z[r][c] < thr) b = fmaxf(b, z[r][c]);
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == src) { lo = a; hi = b; }
    }
    if (valid) {
        float zmin = 0.0f, zmax = 0.0f, width = 0.0f;
        if (act && lo < px.thr) {
            zmin = lo;
            zmax = hi;
            width = penumbra_width(zf, zmin, zmax, g.radius);
        }
        blocker_out[p] = zmin;
        blocker_out[npx + p] = zmax;
        blocker_out[2 * npx + p] = width;
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
    features_kernel<<<blocks, threads, 0, stream>>>(g, feat, texel_out, hard_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !blocker_out) return e;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(blocker_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlockerSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((g.W + kBTile - 1) / kBTile, (g.H + kBTile - 1) / kBTile);
    blocker_kernel<<<grid, kBTile * kBTile, kBlockerSmem, stream>>>(g, blocker_out);
    return cudaGetLastError();
}

}  // namespace nsm
