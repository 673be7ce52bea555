// Per-frame analysis on the device:
//   * the temporal-instability metric of Eq. 3 (Sec. 3.4) between two
//     consecutive frames: every pixel's world position is reprojected into
//     the previous frame's pinhole camera, pixels that fail the depth / normal
//     comparison are rejected, and exp(alpha |I_t(p) - I_{t-1}(m(p))|) - 1 is
//     summed over the rest;
//   * the histogram of screen-space penumbra widths (Sec. 3.6) from the
//     blocker search's spherical-occluder width, whose 95th percentile sets
//     the network depth l = ceil(log2(p_w / 3)).
// Reprojection, acceptance and the pixel difference are binary32 with a fixed
// operation order and no contraction, so the accepted-pixel count is
// reproducible exactly; sums are accumulated in FP64.  Both kernels are
// HBM-bound grid-stride loops (one or two G-buffers read per pixel), reduced
// per warp, then per block, with one global atomic per block.
#include <cmath>

#include "nsm_internal.h"

namespace nsm {

struct PinholeCam {
    float C[3], f[3], r[3], u[3];
    float th, asp;
};

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, const float* b) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a0, b[0]), __fmul_rn(a1, b[1])), __fmul_rn(a2, b[2]));
}

__global__ void __launch_bounds__(256) instability_kernel(int H, int W, const float* __restrict__ vis,
                                                          const float* __restrict__ vis_prev,
                                                          const float4* __restrict__ pos,
                                                          const float4* __restrict__ nrm,
                                                          const float4* __restrict__ pos_prev,
                                                          const float4* __restrict__ nrm_prev, PinholeCam cam,
                                                          float alpha, double* sum_out,
                                                          unsigned long long* count_out) {
    const size_t npx = static_cast<size_t>(H) * W;
    const float Wf = static_cast<float>(W), Hf = static_cast<float>(H);
    const float tha = __fmul_rn(cam.th, cam.asp);
    double s = 0.0;
    unsigned long long c = 0;
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < npx;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float4 P = __ldg(pos + p);
        if (!(P.w > 0.f)) continue;
        const float v0 = __fsub_rn(P.x, cam.C[0]), v1 = __fsub_rn(P.y, cam.C[1]), v2 = __fsub_rn(P.z, cam.C[2]);
        const float z = dot3_rn(v0, v1, v2, cam.f);
        if (!(z > 0.f)) continue;
        const float nx = __fdiv_rn(dot3_rn(v0, v1, v2, cam.r), __fmul_rn(z, tha));
        const float ny = __fdiv_rn(dot3_rn(v0, v1, v2, cam.u), __fmul_rn(z, cam.th));
        const float fi = floorf(__fmul_rn(__fadd_rn(__fmul_rn(nx, 0.5f), 0.5f), Wf));
        const float fj = floorf(__fmul_rn(__fsub_rn(0.5f, __fmul_rn(ny, 0.5f)), Hf));
        if (!(fi >= 0.f && fi < Wf && fj >= 0.f && fj < Hf)) continue;
        const size_t m = static_cast<size_t>(fj) * W + static_cast<size_t>(fi);
        const float dp = __ldg(pos_prev + m).w;
        if (!(dp > 0.f) || !(fabsf(__fsub_rn(dp, z)) <= __fmul_rn(0.01f, z))) continue;
        const float4 Nc = __ldg(nrm + p), Np = __ldg(nrm_prev + m);
        const float nn[3] = {Np.x, Np.y, Np.z};
        if (!(dot3_rn(Nc.x, Nc.y, Nc.z, nn) >= 0.9f)) continue;
        const float D = fabsf(__fsub_rn(__ldg(vis + p), __ldg(vis_prev + m)));
        s += static_cast<double>(expm1f(alpha * D));
        ++c;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    __shared__ double ws[8];
    __shared__ unsigned long long wc[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        ws[warp] = s;
        wc[warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        unsigned long long bc = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
            bs += ws[w];
            bc += wc[w];
        }
        if (bc) {
            atomicAdd(sum_out, bs);
            atomicAdd(count_out, bc);
        }
    }
}

// Screen-space width w H / (2 d tan(fovy / 2)) of every pixel with a blocker
// (z_max > 0), binned by floor(w / bin_px) (negative widths in bin 0, the last
// bin open-ended); a shared-memory histogram per block, added to the output.
__global__ void __launch_bounds__(256) penumbra_hist_kernel(int H, int W, const float* __restrict__ blocker,
                                                            const float4* __restrict__ pos, float tan_half_fovy,
                                                            float bin_px, int nbins, unsigned int* hist) {
    extern __shared__ unsigned int sh[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const size_t npx = static_cast<size_t>(H) * W;
    const float Hf = static_cast<float>(H);
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < npx;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float zmax = __ldg(blocker + npx + p);
        const float d = __ldg(pos + p).w;
        if (!(zmax > 0.f) || !(d > 0.f)) continue;
        const float w = __fdiv_rn(__fmul_rn(__ldg(blocker + 2 * npx + p), Hf), __fmul_rn(__fmul_rn(2.f, d), tan_half_fovy));
        const float fb = floorf(__fdiv_rn(w, bin_px));
        const int b = fb < 0.f ? 0 : (fb >= static_cast<float>(nbins - 1) ? nbins - 1 : static_cast<int>(fb));
        atomicAdd(sh + b, 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + b, sh[b]);
}

static unsigned grid_for(size_t items) {
    const size_t cap = static_cast<size_t>(num_sms()) * 8;
    const size_t b = (items + 255) / 256;
    return static_cast<unsigned>(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace nsm

using namespace nsm;

extern "C" {

nsm_status nsm_temporal_instability(int H, int W, const float* vis, const float* vis_prev, const float* pos4,
                                    const float* nrm4, const float* pos4_prev, const float* nrm4_prev,
                                    const float* cam_prev, float alpha, double* sum_inout,
                                    unsigned long long* count_inout, void* stream) {
    if (H < 0 || W < 0 || !cam_prev || !(alpha >= 0.f))
        return fail(NSM_ERR_INVALID_ARG, "H, W must be >= 0, cam_prev non-NULL and alpha >= 0");
    const size_t npx = static_cast<size_t>(H) * W;
    if (npx == 0) return NSM_OK;
    nsm_status s;
    if ((s = check_dev_ptr(vis, "vis", 4)) != NSM_OK || (s = check_dev_ptr(vis_prev, "vis_prev", 4)) != NSM_OK ||
        (s = check_dev_ptr(pos4, "pos4", 16)) != NSM_OK || (s = check_dev_ptr(nrm4, "nrm4", 16)) != NSM_OK ||
        (s = check_dev_ptr(pos4_prev, "pos4_prev", 16)) != NSM_OK ||
        (s = check_dev_ptr(nrm4_prev, "nrm4_prev", 16)) != NSM_OK ||
        (s = check_dev_ptr(sum_inout, "sum_inout", 8)) != NSM_OK ||
        (s = check_dev_ptr(count_inout, "count_inout", 8)) != NSM_OK)
        return s;
    PinholeCam c{};
    for (int k = 0; k < 3; ++k) {
        c.C[k] = cam_prev[k];
        c.f[k] = cam_prev[3 + k];
        c.r[k] = cam_prev[6 + k];
        c.u[k] = cam_prev[9 + k];
    }
    c.th = cam_prev[12];
    c.asp = cam_prev[13];
    instability_kernel<<<grid_for(npx), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        H, W, vis, vis_prev, reinterpret_cast<const float4*>(pos4), reinterpret_cast<const float4*>(nrm4),
        reinterpret_cast<const float4*>(pos4_prev), reinterpret_cast<const float4*>(nrm4_prev), c, alpha, sum_inout,
        count_inout);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "temporal_instability launch");
}

nsm_status nsm_penumbra_histogram(int H, int W, const float* blocker, const float* pos4, float tan_half_fovy,
                                  float bin_px, int nbins, uint32_t* hist_inout, void* stream) {
    if (H < 0 || W < 0 || !(tan_half_fovy > 0.f) || !(bin_px > 0.f) || nbins < 1 || nbins > NSM_MAX_PENUMBRA_BINS)
        return fail(NSM_ERR_INVALID_ARG, "H, W >= 0, tan_half_fovy > 0, bin_px > 0, 1 <= nbins <= %d",
                    NSM_MAX_PENUMBRA_BINS);
    const size_t npx = static_cast<size_t>(H) * W;
    if (npx == 0) return NSM_OK;
    nsm_status s;
    if ((s = check_dev_ptr(blocker, "blocker", 4)) != NSM_OK || (s = check_dev_ptr(pos4, "pos4", 16)) != NSM_OK ||
        (s = check_dev_ptr(hist_inout, "hist_inout", 4)) != NSM_OK)
        return s;
    penumbra_hist_kernel<<<grid_for(npx), 256, nbins * sizeof(unsigned int), static_cast<cudaStream_t>(stream)>>>(
        H, W, blocker, reinterpret_cast<const float4*>(pos4), tan_half_fovy, bin_px, nbins, hist_inout);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "penumbra_histogram launch");
}

nsm_status nsm_depth_for_penumbra(const uint32_t* hist, int nbins, float bin_px, float* p95_px, int* levels) {
    if (!hist || nbins < 1 || !(bin_px > 0.f) || !p95_px || !levels)
        return fail(NSM_ERR_INVALID_ARG, "hist, p95_px, levels non-NULL, nbins >= 1, bin_px > 0");
    unsigned long long total = 0;
    for (int b = 0; b < nbins; ++b) total += hist[b];
    *p95_px = 0.f;
    *levels = 1;
    if (total == 0) return NSM_OK;
    // first bin whose cumulative count reaches 95% of the total (20 * cum >= 19 * total)
    unsigned long long cum = 0;
    int k = nbins - 1;
    for (int b = 0; b < nbins; ++b) {
        cum += hist[b];
        if (20ull * cum >= 19ull * total) {
            k = b;
            break;
        }
    }
    const double pw = (k + 1) * static_cast<double>(bin_px);
    *p95_px = static_cast<float>(pw);
    int l = 1;
    while (3.0 * std::ldexp(1.0, l) < pw) ++l;  // smallest l >= 1 with 3 * 2^l >= p_w
    *levels = l;
    return NSM_OK;
}

}  // extern "C"
