// Feature sensitivity (Sec. 3.2, Eq. 1): how much the network output changes
// when one input feature channel is perturbed by Gaussian noise of a tenth of
// that channel's standard deviation, normalised by that noise level:
//     S_i = E[ |phi(f_i + eps_i) - phi(f_i)| ] / (0.1 sigma_i),  eps_i ~ N(0, (0.1 sigma_i)^2)
// (the expectation over pixels, frames and repeated draws; |.| is the reading
// of Eq. 1's expectation, whose signed form is about zero for symmetric
// noise).  The perturbed channel is changed inside the fused gather, so every
// evaluation is one ordinary inference pass.
//
//   nsm_feature_moments  per-channel sums of f and f^2 over a frame's pixels
//                        (FP64, accumulated): sigma_i over a set of frames
//   nsm_sensitivity      the base pass and one perturbed pass per (channel,
//                        draw), accumulating sum |delta phi| / (0.1 sigma_i)
#include "../../include/nsm.h"
#include "nsm_internal.h"
#include "ctx_internal.h"

namespace nsm {

constexpr int kRedThreads = 256;

// block-wide sum of a double (kRedThreads threads), result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    }
    __syncthreads();
    return v;
}

// sums of f_c and f_c^2 (c = 0..3) over the frame's pixels, added to moments[8]
__global__ void __launch_bounds__(kRedThreads) feature_moments_kernel(GatherParams g, double* moments) {
    __shared__ double sh[kRedThreads / 32];
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const size_t n = static_cast<size_t>(g.H) * g.W;
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const PixelGather o = gather_pixel(g, __ldg(g.pos4 + p), __ldg(g.nrm4 + p));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            s[c] += o.f[c];
            s[4 + c] += static_cast<double>(o.f[c]) * o.f[c];
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double t = block_sum(s[k], sh);
        if (threadIdx.x == 0) atomicAdd(moments + k, t);
    }
}

// sum |a - b| / norm over n values, added to *out
__global__ void __launch_bounds__(kRedThreads) abs_diff_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                               size_t n, double inv_norm, double* out) {
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        s += fabs(static_cast<double>(__ldg(a + i)) - static_cast<double>(__ldg(b + i)));
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(out, s * inv_norm);
}

static int red_grid(size_t n) {
    const size_t want = (n + kRedThreads - 1) / kRedThreads;
    const size_t cap = static_cast<size_t>(4) * num_sms();
    return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace nsm

using namespace nsm;

extern "C" {

nsm_status nsm_feature_moments(const nsm_frame* frame, double* moments_inout, void* stream) {
    nsm_status s = check_frame(frame, false);
    if (s != NSM_OK) return s;
    const size_t n = static_cast<size_t>(frame->H) * frame->W;
    if (n == 0) return NSM_OK;
    if ((s = check_dev_ptr(moments_inout, "moments_inout", 8)) != NSM_OK) return s;
    feature_moments_kernel<<<red_grid(n), kRedThreads, 0, static_cast<cudaStream_t>(stream)>>>(make_gather(frame),
                                                                                                moments_inout);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "feature moments kernel");
}

size_t nsm_sensitivity_workspace_bytes(int H, int W) {
    if (H <= 0 || W <= 0) return 0;
    const size_t npx = static_cast<size_t>(H) * W;
    return nsm_infer_workspace_bytes(H, W, NSM_FP32) + 2 * align_up(npx * sizeof(float), 256);
}

nsm_status nsm_sensitivity(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w, nsm_precision precision,
                           const float* noise, int draws, const float* sigma, void* workspace, size_t workspace_bytes,
                           double* s_inout, void* stream) {
    if (!ctx || !w) return fail(NSM_ERR_INVALID_ARG, "ctx and weights must be non-NULL");
    if (precision != NSM_FP32 && precision != NSM_BF16)
        return fail(NSM_ERR_UNSUPPORTED, "the sensitivity runs in the FP32 and BF16 forms");
    if (draws < 1) return fail(NSM_ERR_INVALID_ARG, "draws must be >= 1");
    if (!sigma) return fail(NSM_ERR_INVALID_ARG, "sigma is NULL");
    for (int c = 0; c < 4; ++c)
        if (!(sigma[c] > 0.f) || !finite_all(sigma + c, 1))
            return fail(NSM_ERR_INVALID_ARG, "sigma[%d] must be finite and > 0", c);
    nsm_status s = check_frame(frame, true);
    if (s != NSM_OK) return s;
    const size_t npx = static_cast<size_t>(frame->H) * frame->W;
    if (npx == 0) return NSM_OK;
    if ((s = check_dev_ptr(noise, "noise", 4)) != NSM_OK || (s = check_dev_ptr(s_inout, "s_inout", 8)) != NSM_OK)
        return s;
    const size_t need = nsm_sensitivity_workspace_bytes(frame->H, frame->W);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    const size_t act = nsm_infer_workspace_bytes(frame->H, frame->W, NSM_FP32);
    float* base = reinterpret_cast<float*>(static_cast<char*>(workspace) + act);
    float* pert = reinterpret_cast<float*>(static_cast<char*>(workspace) + act + align_up(npx * sizeof(float), 256));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = infer_impl(ctx, frame, w, precision, workspace, act, base, stream, nullptr, 0.f, 0)) != NSM_OK) return s;
    for (int c = 0; c < 4; ++c) {
        const float scale = 0.1f * sigma[c];
        for (int k = 0; k < draws; ++k) {
            const float* eps = noise + (static_cast<size_t>(k) * 4 + c) * npx;
            if ((s = infer_impl(ctx, frame, w, precision, workspace, act, pert, stream, eps, scale, c)) != NSM_OK)
                return s;
            abs_diff_kernel<<<red_grid(npx), kRedThreads, 0, st>>>(pert, base, npx, 1.0 / scale, s_inout + c);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "sensitivity reduction kernel");
        }
    }
    return NSM_OK;
}

}  // extern "C"
