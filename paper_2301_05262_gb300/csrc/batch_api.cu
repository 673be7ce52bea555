// Batched serving (many views of uneven size per launch), its CUDA-graph
// cache and the tile autotuner (include/nsm.h).
#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx_internal.h"

namespace nsm {

static nsm_status check_views(int n, const nsm_view* views) {
    if (n < 1 || n > kMaxViews) return fail(NSM_ERR_SHAPE, "%d views; 1 to %d per call", n, kMaxViews);
    if (!views) return fail(NSM_ERR_INVALID_ARG, "views is NULL");
    for (int i = 0; i < n; ++i) {
        nsm_status s = check_frame(&views[i].frame, true);
        if (s != NSM_OK) return s;
        if (static_cast<size_t>(views[i].frame.H) * views[i].frame.W == 0)
            return fail(NSM_ERR_SHAPE, "view %d is empty", i);
        if ((s = check_dev_ptr(views[i].vis_out, "view.vis_out", 4)) != NSM_OK) return s;
    }
    return NSM_OK;
}

// Activations of every view, carved from the workspace one after another.
static void carve_views(int n, const nsm_view* views, void* ws, std::vector<Activations>& act,
                        std::vector<GatherParams>& gp, std::vector<float*>& vis) {
    act.resize(n);
    gp.resize(n);
    vis.resize(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const nsm_frame& f = views[i].frame;
        off += activations_bytes(f.H, f.W, 4, &act[i], static_cast<char*>(ws) + off);
        gp[i] = make_gather(&f);
        vis[i] = views[i].vis_out;
    }
}

static std::vector<long long> plan_key(const nsm_ctx* c, int n, const nsm_view* views) {
    std::vector<long long> k;
    k.push_back(n);
    for (int i = 0; i < n; ++i) {
        k.push_back(views[i].frame.H);
        k.push_back(views[i].frame.W);
    }
    for (int s = 0; s < kTcStages; ++s) {
        k.push_back(c->tc_variant[s]);
        k.push_back(c->tc_ctas[s]);
    }
    return k;
}

}  // namespace nsm

using namespace nsm;

void ctx_release_graph(nsm_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_key.clear();
}

extern "C" {

size_t nsm_infer_batched_workspace_bytes(int n, const nsm_view* views) {
    if (n < 1 || n > kMaxViews || !views) return 0;
    size_t t = 0;
    for (int i = 0; i < n; ++i) {
        if (views[i].frame.H <= 0 || views[i].frame.W <= 0) return 0;
        t += activations_bytes(views[i].frame.H, views[i].frame.W, 4, nullptr, nullptr);
    }
    return t;
}

nsm_status nsm_ctx_set_view_timing(nsm_ctx* c, unsigned long long* dev_records) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    nsm_status s;
    if (dev_records && (s = check_dev_ptr(dev_records, "dev_records", 8)) != NSM_OK) return s;
    c->view_timing = dev_records;
    ctx_release_graph(c);  // the kernels' argument changes
    return NSM_OK;
}

nsm_status nsm_ctx_set_graph(nsm_ctx* c, int enable) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    c->use_graph = enable ? 1 : 0;
    if (!enable) ctx_release_graph(c);
    return NSM_OK;
}

int nsm_ctx_graph_replays(nsm_ctx* c) { return c ? c->graph_launches : 0; }

nsm_status nsm_infer_batched(nsm_ctx* c, int n, const nsm_view* views, const nsm_weights* w, void* workspace,
                             size_t workspace_bytes, void* stream) {
    if (!c || !w) return fail(NSM_ERR_INVALID_ARG, "ctx and weights must be non-NULL");
    if (w->topology != NSM_TOPO_LEVELS3) return fail(NSM_ERR_UNSUPPORTED, "batched calls take 3-level weights");
    nsm_status s = check_views(n, views);
    if (s != NSM_OK) return s;
    const size_t need = nsm_infer_batched_workspace_bytes(n, views);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<Activations> act;
    std::vector<GatherParams> gp;
    std::vector<float*> vis;
    carve_views(n, views, workspace, act, gp, vis);
    TcBatch b[kTcStages];
    tc_make_batches(gp.data(), act.data(), vis.data(), n, w->d_params, w->d_bf16, c->d_err, b);
    b[0].timing = b[kTcStages - 1].timing = c->view_timing;
    cudaError_t e;
    if (!c->use_graph) {
        for (int k = 0; k < kTcStages; ++k)
            if ((e = tc_launch_stage(k, c->tc_variant[k], b[k], c->tc_ctas[k], st)) != cudaSuccess)
                return cuda_fail(e, "stage launch");
        return NSM_OK;
    }
    const std::vector<long long> key = plan_key(c, n, views);
    if (key != c->graph_key) {
        // new plan: make sure every kernel is set up (attributes) outside the
        // capture, then capture the five stage launches into a graph
        ctx_release_graph(c);
        for (int k = 0; k < kTcStages; ++k) tc_stage_occupancy(k, c->tc_variant[k]);
        cudaStream_t cap;
        if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
        TcBatch warm[kTcStages];
        std::memcpy(warm, b, sizeof(b));
        for (int k = 0; k < kTcStages && e == cudaSuccess; ++k)  // first launches (function attributes) uncaptured
            e = tc_launch_stage(k, c->tc_variant[k], warm[k], c->tc_ctas[k], cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cap);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < kTcStages && e == cudaSuccess; ++k)
            e = tc_launch_stage(k, c->tc_variant[k], b[k], c->tc_ctas[k], cap);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "graph capture"); }
        // find the kernel node of each stage by its function
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int found = 0;
        for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            cudaGraphNodeGetType(nodes[i], &t);
            if (t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams p{};
            cudaGraphKernelNodeGetParams(nodes[i], &p);
            for (int k = 0; k < kTcStages; ++k)
                if (p.func == tc_stage_kernel(k, c->tc_variant[k])) {
                    c->graph_nodes[k] = nodes[i];
                    c->graph_params[k] = p;
                    ++found;
                }
        }
        if (found != kTcStages) { cudaGraphDestroy(g); return fail(NSM_ERR_CUDA, "graph capture: %d kernel nodes", found); }
        cudaGraphExec_t ex = nullptr;
        if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "graph instantiate"); }
        c->graph = g;
        c->graph_exec = ex;
        c->graph_key = key;
        c->graph_launches = 0;
    } else {
        // same plan: point the captured kernel nodes at this call's job tables
        for (int k = 0; k < kTcStages; ++k) {
            // the tile tables are a pure function of the plan; refill them for the job copy
            TcBatch& bk = b[k];
            if ((e = tc_prepare_stage(k, c->tc_variant[k], bk)) != cudaSuccess) return cuda_fail(e, "stage set-up");
            cudaKernelNodeParams p = c->graph_params[k];
            void* args[1] = {&bk};
            p.kernelParams = args;
            p.extra = nullptr;
            if ((e = cudaGraphExecKernelNodeSetParams(c->graph_exec, c->graph_nodes[k], &p)) != cudaSuccess)
                return cuda_fail(e, "graph node update");
        }
    }
    if ((e = cudaGraphLaunch(c->graph_exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
    c->graph_launches += 1;
    return NSM_OK;
}

nsm_status nsm_autotune(nsm_ctx* c, int n, const nsm_view* views, const nsm_weights* w, void* workspace,
                        size_t workspace_bytes, int reps, void* stream) {
    if (!c || !w) return fail(NSM_ERR_INVALID_ARG, "ctx and weights must be non-NULL");
    if (w->topology != NSM_TOPO_LEVELS3) return fail(NSM_ERR_UNSUPPORTED, "batched calls take 3-level weights");
    nsm_status s = check_views(n, views);
    if (s != NSM_OK) return s;
    const size_t need = nsm_infer_batched_workspace_bytes(n, views);
    if (!workspace || workspace_bytes < need)
        return fail(NSM_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
    if ((s = check_dev_ptr(workspace, "workspace", 256)) != NSM_OK) return s;
    if (reps < 1) reps = 3;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<Activations> act;
    std::vector<GatherParams> gp;
    std::vector<float*> vis;
    carve_views(n, views, workspace, act, gp, vis);
    TcBatch b[kTcStages];
    tc_make_batches(gp.data(), act.data(), vis.data(), n, w->d_params, w->d_bf16, c->d_err, b);
    cudaError_t e = cudaSuccess;
    // one pass with the current plan so that every stage's input holds real data
    for (int k = 0; k < kTcStages && e == cudaSuccess; ++k) e = tc_launch_stage(k, c->tc_variant[k], b[k], c->tc_ctas[k], st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < kTcStages && e == cudaSuccess; ++k) {
        float best = 1e30f;
        int bv = c->tc_variant[k], bc = c->tc_ctas[k];
        for (int v = 0; v < tc_stage_variants(k) && e == cudaSuccess; ++v) {
            const int occ = tc_stage_occupancy(k, v);
            for (int cta = 1; cta <= occ && e == cudaSuccess; ++cta) {
                e = tc_launch_stage(k, v, b[k], cta, st);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = tc_launch_stage(k, v, b[k], cta, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                if (e == cudaSuccess && ms < best) { best = ms; bv = v; bc = cta; }
            }
        }
        c->tc_variant[k] = bv;
        c->tc_ctas[k] = bc;
        c->tc_ms[k] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    ctx_release_graph(c);  // the plan changed
    return NSM_OK;
}

nsm_status nsm_autotune_report(nsm_ctx* c, int* rows_out, int* ctas_out, float* ms_out) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    for (int k = 0; k < kTcStages; ++k) {
        if (rows_out) rows_out[k] = tc_stage_rows(k, c->tc_variant[k]);
        if (ctas_out) ctas_out[k] = c->tc_ctas[k];
        if (ms_out) ms_out[k] = c->tc_ms[k];
    }
    return NSM_OK;
}

nsm_status nsm_autotune_report_warps(nsm_ctx* c, int* epilogue_warps_out, int* producer_warps_out) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    for (int k = 0; k < kTcStages; ++k) {
        int pw = 0;
        const int ew = tc_stage_warps(k, c->tc_variant[k], &pw);
        if (epilogue_warps_out) epilogue_warps_out[k] = ew;
        if (producer_warps_out) producer_warps_out[k] = pw;
    }
    return NSM_OK;
}

int nsm_plan_variants(int stage) { return tc_stage_variants(stage); }

nsm_status nsm_plan_set(nsm_ctx* c, int stage, int variant, int ctas_per_sm) {
    if (!c) return fail(NSM_ERR_INVALID_ARG, "ctx is NULL");
    if (stage < 0 || stage >= kTcStages || variant < 0 || variant >= tc_stage_variants(stage) || ctas_per_sm < 0)
        return fail(NSM_ERR_INVALID_ARG, "stage 0..%d, variant 0..nsm_plan_variants(stage)-1, ctas_per_sm >= 0",
                    kTcStages - 1);
    c->tc_variant[stage] = variant;
    c->tc_ctas[stage] = ctas_per_sm;
    c->tc_ms[stage] = 0.f;
    ctx_release_graph(c);  // the plan changed
    return NSM_OK;
}

nsm_status nsm_autotune_report_order(nsm_ctx* c, int* mma_order_out) {
    if (!c || !mma_order_out) return fail(NSM_ERR_INVALID_ARG, "ctx and mma_order_out must be non-NULL");
    for (int k = 0; k < kTcStages; ++k) mma_order_out[k] = tc_stage_order(k, c->tc_variant[k]);
    return NSM_OK;
}

}  // extern "C"
