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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <string>

#include "../../include/nsm.h"
#include "nsm_internal.h"

namespace nsm {

constexpr size_t kStaticMaxPixels = 512 * 512;
// 80 bytes per pixel of FP32 activations (16 + 32 + 16 channels at half
// resolution, 32 + 32 at quarter resolution) plus 256-byte alignment of the
// five buffers.
constexpr size_t kStaticScratchBytes = 80 * kStaticMaxPixels + 5 * 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch in the current context.  In host code
// the array's name is only a host-side stand-in, so kernels must get this
// address, never the symbol itself.  It is looked up on every call (a host-side
// table lookup that allocates nothing): after a device reset, or once the
// primary context has been released and made again, the module is loaded anew
// and the array can sit at another address, so a cached value could go stale.
static cudaError_t static_scratch_address(void** out) {
    *out = nullptr;
    return cudaGetSymbolAddress(out, g_static_scratch);
}

// The allocation that holds p must extend at least `bytes` past p.  Buffers
// from a caching allocator are checked against the block they were carved
// from, which still keeps every access inside mapped memory.
// The driver function is resolved through the runtime, so the library does
// not link libcuda itself (it loads on machines without a driver, where only
// its host-side checks run).
static nsm_status check_extent(const void* p, size_t bytes, const char* name) {
    static const PFN_cuMemGetAddressRange_v3020 get_range = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 3020, cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(fn)
                                                                     : nullptr;
    }();
    if (!get_range) return fail(NSM_ERR_CUDA, "cannot resolve cuMemGetAddressRange");
    CUdeviceptr base = 0;
    size_t size = 0;
    CUresult r = get_range(&base, &size, reinterpret_cast<CUdeviceptr>(p));
    if (r != CUDA_SUCCESS) return fail(NSM_ERR_INVALID_ARG, "%s: cannot query its allocation (CUresult %d)", name, r);
    const size_t avail = static_cast<size_t>(base + size - reinterpret_cast<CUdeviceptr>(p));
    if (avail < bytes)
        return fail(NSM_ERR_INVALID_ARG, "%s: its allocation holds %zu bytes from this address, %zu needed", name, avail,
                    bytes);
    return NSM_OK;
}

}  // namespace nsm

using namespace nsm;

extern "C" nsm_status nsm_infer_fp32_static(const nsm_frame* f, const float* dev_params, float* vis_out,
                                            void* stream) {
    // sizes and light / camera values first: no CUDA call before these
    nsm_status s = check_frame_host(f, true);
    if (s != NSM_OK) return s;
    const size_t npx = static_cast<size_t>(f->H) * f->W;
    if (npx > kStaticMaxPixels)
        return fail(NSM_ERR_SHAPE,
                    "view of %d x %d = %zu pixels exceeds the static scratch limit of %zu pixels; use nsm_infer "
                    "with a workspace",
                    f->H, f->W, npx, kStaticMaxPixels);
    if (npx == 0) return NSM_OK;
    if ((s = check_device()) != NSM_OK) return s;
    if ((s = check_frame(f, true)) != NSM_OK) return s;
    if ((s = check_dev_ptr(dev_params, "dev_params", 4)) != NSM_OK) return s;
    if ((s = check_dev_ptr(vis_out, "vis_out", 4)) != NSM_OK) return s;
    const LayerOffsets lo = layer_offsets();
    if ((s = check_extent(dev_params, lo.total * sizeof(float), "dev_params")) != NSM_OK) return s;
    if ((s = check_extent(vis_out, npx * sizeof(float), "vis_out")) != NSM_OK) return s;
    if ((s = check_extent(f->pos4, npx * 16, "frame.pos4")) != NSM_OK) return s;
    if ((s = check_extent(f->nrm4, npx * 16, "frame.nrm4")) != NSM_OK) return s;
    if ((s = check_extent(f->sm, static_cast<size_t>(f->Hs) * f->Ws * sizeof(float), "frame.sm")) != NSM_OK)
        return s;

    void* scratch = nullptr;
    cudaError_t e = static_scratch_address(&scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    Activations act{};
    if (activations_bytes(f->H, f->W, 4, &act, scratch) > kStaticScratchBytes)
        return fail(NSM_ERR_SHAPE, "internal: activations exceed the static scratch");
    e = launch_infer_fp32(make_gather(f), dev_params, act, vis_out, static_cast<cudaStream_t>(stream), StageEvents{});
    if (e != cudaSuccess) return cuda_fail(e, "inference kernel launch");
    return NSM_OK;
}
