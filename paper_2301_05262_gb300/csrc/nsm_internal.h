// Internal (host-side) declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "nsm_common.cuh"

namespace nsm {

// Device staging slots of nsm_infer_host_sequence (frames in flight).
constexpr int kMaxHostSlots = 3;

// Canonical layer table of the 3-level network (Sec. 3.5): offsets of each
// layer's OIHW weights and bias in the canonical parameter vector.
enum Layer { ENC0_3, ENC0_1, ENC1_3, ENC1_1, BOTT_3, BOTT_1, DEC1_3, DEC1_1, DEC0_3, DEC0_1, HEAD, NUM_LAYERS };

struct LayerShape { int cin, cout, k; };
constexpr LayerShape kLayers[NUM_LAYERS] = {
    {4, 16, 3}, {16, 16, 1}, {16, 32, 3}, {32, 32, 1}, {32, 64, 3}, {64, 32, 1},
    {32, 32, 3}, {32, 16, 1}, {16, 16, 3}, {16, 16, 1}, {16, 1, 1}};

struct LayerOffsets { size_t w[NUM_LAYERS]; size_t b[NUM_LAYERS]; size_t total; };
LayerOffsets layer_offsets();
// Space-to-depth topology (Sec. 3.5): the level-0 layers removed (offsets
// SIZE_MAX) and the head 16 -> 4 (stored at index HEAD).
LayerOffsets layer_offsets_s2d();
constexpr int kS2dHeadOut = 4;

int num_sms();
// CTAs of `func` (block of `threads`, `dyn_smem` bytes of dynamic shared
// memory) that fit on one SM of the current device, counted from the
// function's registers and shared memory against the SM's registers, shared
// memory (less the per-block reservation), threads and block slots.  The
// tcgen05 kernels size their grids with this: the runtime's occupancy query
// answers one CTA per SM for them where several fit.
int resident_ctas_per_sm(const void* func, int threads, size_t dyn_smem);
// The library's stream-ordered scratch pool for the current device.
cudaError_t scratch_pool(cudaMemPool_t* out);

// Message returned by nsm_last_error() on this thread.
void set_last_error(const std::string& msg);

}  // namespace nsm
#include "../../include/nsm.h"
namespace nsm {
// Host-side validation helpers of the C ABI (nsm_api.cu).
nsm_status fail(nsm_status s, const char* fmt, ...);
nsm_status cuda_fail(cudaError_t e, const char* what);
nsm_status check_device();
nsm_status check_dev_ptr(const void* p, const char* name, size_t align, bool nullable = false);
bool finite_all(const float* v, int n);
// Sizes and light / camera values only (no CUDA call); check_frame adds the
// device-pointer checks of the G-buffer and the map.
nsm_status check_frame_host(const nsm_frame* f, bool need_mult4);
nsm_status check_frame(const nsm_frame* f, bool need_mult4);
GatherParams make_gather(const nsm_frame* f);
// nsm_infer with an optional feature perturbation (feat_eps null: none; see GatherParams)
nsm_status infer_impl(nsm_ctx* ctx, const nsm_frame* frame, const nsm_weights* w, nsm_precision precision,
                      void* workspace, size_t workspace_bytes, float* vis_out, void* stream, const float* feat_eps,
                      float eps_scale, int eps_ch);
size_t align_up(size_t v, size_t a);

// Activation buffers of one inference, carved out of the caller's workspace.
struct Activations {
    // FP32 [..][C], or BF16 hi + lo pairs [..][2][C]: 4 bytes per channel
    void* e0;   // [H/2][W/2][16]  pooled level-0 encoder output
    void* s1;   // [H/2][W/2][32]  level-1 encoder output (decoder skip)
    void* p1;   // [H/4][W/4][32]  pooled level-1 encoder output
    void* bo;   // [H/4][W/4][32]  bottleneck output
    void* d1;   // [H/2][W/2][16]  level-1 decoder output
};
size_t activations_bytes(int H, int W, size_t elem_bytes, Activations* carve, void* base);

// Optional per-kernel event recording (profiling hook of nsm_ctx).
struct StageEvents {
    cudaEvent_t* ev = nullptr;
    int n = 0;
    cudaStream_t stream = nullptr;
    inline void rec(int i) const {
        if (ev && i < n) cudaEventRecord(ev[i], stream);
    }
};

// table_ws: >= 16 Ws Hs bytes, 16-byte aligned, for the blocker search's
// tables; null takes stream-ordered scratch from scratch_pool
cudaError_t launch_features(const GatherParams& g, float* feat, int32_t* texel_out, uint32_t* hard_out,
                            float* blocker_out, void* table_ws, cudaStream_t stream);

constexpr int kInferKernelsFp32 = 5;
extern const char* const kInferKernelNamesFp32[kInferKernelsFp32];
cudaError_t launch_infer_fp32(const GatherParams& g, const float* params, const Activations& act,
                              float* vis, cudaStream_t stream, const StageEvents& se);

// Packed BF16 weight images for the tensor-core form (shared-memory layout of
// each layer's B operand), built on the device from the canonical FP32 vector.
struct PackDescHost { int kind, cin, cout; size_t w_off; size_t img_off; size_t count; };
struct BF16Images {
    PackDescHost desc[NUM_LAYERS];
    int n;
    size_t img_off[NUM_LAYERS];  // element offset of each layer's image (head has none)
    size_t total;                // elements (uint16)
};
BF16Images bf16_images(bool s2d = false);
size_t pack_desc_bytes();
cudaError_t launch_pack_bf16(const float* params, uint16_t* img, const void* dev_descs, int ndesc,
                             cudaStream_t stream);

// E4M3 weight images + per-output-channel scales of the FP8 form (pack_fp8.cu).
struct F8Images {
    size_t img_off[NUM_LAYERS];    // byte offset of each layer's image (head has none)
    size_t scale_off[NUM_LAYERS];  // offset of each layer's scales (one per output channel)
    size_t img_bytes;
    size_t scales;
};
F8Images fp8_images();
cudaError_t launch_pack_fp8(const float* params, uint8_t* img, float* scales, cudaStream_t stream);

constexpr int kInferKernelsFp8 = 5;
extern const char* const kInferKernelNamesFp8[kInferKernelsFp8];
cudaError_t launch_infer_fp8(const GatherParams& g, const float* params, const uint8_t* img, const float* scales,
                             const Activations& act, float* vis, int* err, cudaStream_t stream,
                             const StageEvents& se);

// Space-to-depth topology, BF16 form: gather + 2x2 flattening, enc1, bottleneck,
// dec1 with the 4-channel head, 2x2 recombination (5 launches).
constexpr int kInferKernelsS2d = 5;
extern const char* const kInferKernelNamesS2d[kInferKernelsS2d];
cudaError_t launch_s2d_features(const GatherParams& g, uint16_t* out, cudaStream_t stream);
cudaError_t launch_s2d_output(const float* o4, int H, int W, float* vis, cudaStream_t stream);
cudaError_t launch_infer_s2d_bf16(const GatherParams& g, const float* params, const uint16_t* img,
                                  const Activations& act, float* vis, int* err, cudaStream_t stream,
                                  const StageEvents& se);

constexpr int kInferKernelsBf16 = 5;
extern const char* const kInferKernelNamesBf16[kInferKernelsBf16];
cudaError_t launch_infer_bf16(const GatherParams& g, const float* params, const uint16_t* img,
                              const Activations& act, float* vis, int* err, cudaStream_t stream,
                              const StageEvents& se, const int* variant, const int* ctas);

}  // namespace nsm
