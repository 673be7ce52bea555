// nsm_infer_fp32_static: FP32 inference that allocates nothing and takes no
// workspace.  For callers that own only their input and output buffers and
// may not allocate device memory themselves -- e.g. a renderer's per-frame
// loop or a plug-in running under a host engine that forbids device
// allocation after start-up (cudaMalloc can synchronise the device and stall
// a frame) and hands the plug-in nothing but the frame's buffers.
//
// The level activations live in one file-scope device array of fixed size,
// sized for views of at most kStaticMaxPixels pixels.  Every GPU that loads
// the library holds this array until the process exits.  All calls share it:
// two calls whose work overlaps on the GPU (different streams, or different
// host threads without ordering) race on it.  Each call overwrites every
// activation element before reading it, so nothing needs clearing between
// calls.
#include <cstring>
#include <mutex>

#include "../../include/nsm.h"
#include "nsm_internal.h"

namespace nsm {

constexpr size_t kStaticMaxPixels = 512 * 512;
// 80 bytes per pixel of FP32 activations (16 + 32 + 16 channels at half
// resolution, 32 + 32 at quarter resolution) plus 256-byte alignment of the
// five buffers.
constexpr size_t kStaticScratchBytes = 80 * kStaticMaxPixels + 5 * 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so kernels must get
// this address, never the symbol itself.
static std::mutex g_static_mu;
static void* g_static_addr[64] = {nullptr};

static cudaError_t static_scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

static nsm_status static_check_ptr(const void* p, const char* name, size_t align, int dev) {
    if (!p) {
        set_last_error(std::string(name) + " is NULL");
        return NSM_ERR_INVALID_ARG;
    }
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        set_last_error(std::string(name) + ": cannot query pointer");
        return NSM_ERR_INVALID_ARG;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
        set_last_error(std::string(name) + " is not device memory of the current device");
        return NSM_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(p) % align) {
        set_last_error(std::string(name) + " is misaligned");
        return NSM_ERR_ALIGNMENT;
    }
    return NSM_OK;
}

}  // namespace nsm

using namespace nsm;

extern "C" nsm_status nsm_infer_fp32_static(const nsm_frame* f, const float* dev_params, float* vis_out,
                                            void* stream) {
    if (!f) { set_last_error("frame is NULL"); return NSM_ERR_INVALID_ARG; }
    if (f->H < 0 || f->W < 0 || (f->H % 4) || (f->W % 4)) {
        set_last_error("view size must be non-negative multiples of 4");
        return NSM_ERR_SHAPE;
    }
    const size_t npx = static_cast<size_t>(f->H) * f->W;
    if (npx > kStaticMaxPixels) {
        set_last_error("view of " + std::to_string(f->H) + " x " + std::to_string(f->W) + " = " +
                       std::to_string(npx) + " pixels exceeds the static scratch limit of " +
                       std::to_string(kStaticMaxPixels) + " pixels; use nsm_infer with a workspace");
        return NSM_ERR_SHAPE;
    }
    if (f->Hs < 1 || f->Ws < 1 || f->Hs > 16384 || f->Ws > 16384) {
        set_last_error("shadow map size outside [1, 16384]");
        return NSM_ERR_SHAPE;
    }
    if (npx == 0) return NSM_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) { set_last_error("no usable CUDA device"); return NSM_ERR_DEVICE; }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) { set_last_error("this library is built for sm_103a only"); return NSM_ERR_DEVICE; }
    nsm_status s;
    if ((s = static_check_ptr(f->pos4, "frame.pos4", 16, dev)) != NSM_OK) return s;
    if ((s = static_check_ptr(f->nrm4, "frame.nrm4", 16, dev)) != NSM_OK) return s;
    if ((s = static_check_ptr(f->sm, "frame.sm", 4, dev)) != NSM_OK) return s;
    if ((s = static_check_ptr(dev_params, "dev_params", 4, dev)) != NSM_OK) return s;
    if ((s = static_check_ptr(vis_out, "vis_out", 4, dev)) != NSM_OK) return s;

    void* scratch = nullptr;
    e = static_scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        return NSM_ERR_CUDA;
    }
    Activations act{};
    if (activations_bytes(f->H, f->W, 4, &act, scratch) > kStaticScratchBytes) {
        set_last_error("internal: activations exceed the static scratch");
        return NSM_ERR_SHAPE;
    }
    GatherParams g{};
    std::memcpy(g.M, f->light.view_proj, sizeof(g.M));
    for (int k = 0; k < 3; ++k) { g.L[k] = f->light.pos[k]; g.C[k] = f->camera.pos[k]; }
    g.r_hat = f->light.r_hat;
    g.z_far = f->light.z_far;
    g.beta = f->light.bias;
    g.radius = f->light.radius;
    g.tan_half_fov = f->light.tan_half_fov;
    g.Ws = f->Ws; g.Hs = f->Hs;
    g.Ws_f = static_cast<float>(f->Ws); g.Hs_f = static_cast<float>(f->Hs);
    g.half_Ws = 0.5f * static_cast<float>(f->Ws);
    g.H = f->H; g.W = f->W;
    g.pos4 = reinterpret_cast<const float4*>(f->pos4);
    g.nrm4 = reinterpret_cast<const float4*>(f->nrm4);
    g.sm = f->sm;
    e = launch_infer_fp32(g, dev_params, act, vis_out, static_cast<cudaStream_t>(stream), StageEvents{});
    if (e != cudaSuccess) {
        set_last_error(std::string("inference kernel launch: ") + cudaGetErrorString(e));
        return NSM_ERR_CUDA;
    }
    return NSM_OK;
}
