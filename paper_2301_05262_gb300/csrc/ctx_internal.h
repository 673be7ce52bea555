// Definitions of the opaque handles of the C ABI (shared by the API files).
#pragma once

#include <vector>

#include "nsm_internal.h"
#include "tc_stage.h"

// Context: device error word, profiling hook, tensor-core tile plan (set by
// the autotuner) and the cached CUDA graph of the batched launch.
struct nsm_ctx {
    int device;
    int* d_err;                              // device error word (bounded waits that gave up)
    std::vector<cudaEvent_t> stage_events;   // profiling hook (caller-owned events)
    int tc_variant[nsm::kTcStages];          // tile variant per stage
    int tc_ctas[nsm::kTcStages];             // CTAs per SM per stage (0 = as many as fit)
    float tc_ms[nsm::kTcStages];             // autotuned stage times (ms), 0 if not tuned
    // CUDA graph of nsm_infer_batched, keyed by the batch plan
    int use_graph;
    std::vector<long long> graph_key;
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    cudaGraphNode_t graph_nodes[nsm::kTcStages];
    cudaKernelNodeParams graph_params[nsm::kTcStages];
    int graph_launches;                      // replays of the cached graph (for tests)
    unsigned long long* view_timing;         // per-view completion records of nsm_infer_batched (null: off)
    // nsm_infer_host_sequence: copy streams and per-slot events (created on first use)
    cudaStream_t h2d_stream, d2h_stream;
    cudaEvent_t slot_h2d[nsm::kMaxHostSlots], slot_inf[nsm::kMaxHostSlots], slot_d2h[nsm::kMaxHostSlots];
    bool slots_ready;
};

struct nsm_weights {
    int device;
    int topology;      // nsm_topology
    float* d_params;   // canonical FP32 vector (nsm_param_count floats)
    uint16_t* d_bf16;  // packed BF16 images (tensor-core form)
    void* d_descs;     // packing table
    int ndesc;
    uint8_t* d_fp8;        // E4M3 images (FP8 form)
    float* d_fp8_scales;   // their per-output-channel scales
};

void ctx_release_graph(nsm_ctx* c);
void ctx_release_host_slots(nsm_ctx* c);
