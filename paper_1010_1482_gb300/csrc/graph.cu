// Repeated evaluations and tuning: the C ABI's gbfmm_graph_* (one uniform-tree evaluation
// captured into a CUDA graph and replayed) and gbfmm_tune_leaf (leaf-size autotuner).
//
// A time-stepping N-body code evaluates the same number of particles in the same buffers at
// every step; the uniform-tree evaluation never synchronises with the host, so its launches can
// be captured once and replayed with a single graph launch.  The autotuner times one evaluation
// of the caller's particles per candidate leaf size (the leaf size moves work between the near
// field and the far field) and returns the fastest.
#include <cuda_runtime.h>

#include <cfloat>

#include "context.h"
#include "gbfmm.h"

struct gbfmm_graph {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using gbfmm::cuda_fail;
using gbfmm::fail;

extern "C" {

int gbfmm_graph_create(gbfmm_graph **out, gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq,
                       float *d_out, void *d_workspace, size_t workspace_bytes)
{
    if (!out || !ctx || !prm) return GBFMM_EINVAL;
    *out = nullptr;
    if (prm->tree != GBFMM_TREE_UNIFORM) return fail(ctx, GBFMM_EUNSUPPORTED, "graphs capture uniform-tree evaluations");
    gbfmm_params p = *prm;
    p.flags &= ~GBFMM_FLAG_STAGE_TIMING;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaStreamCreate");
    // one eager evaluation builds the order's operator tables and validates the arguments
    int rc = gbfmm_evaluate(ctx, &p, n, d_xyzq, d_out, d_workspace, workspace_bytes, s);
    if (rc == GBFMM_OK) rc = gbfmm_sync_status(ctx, s);
    cudaGraph_t graph = nullptr;
    if (rc == GBFMM_OK) {
        if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            rc = cuda_fail(ctx, e, "cudaStreamBeginCapture");
        } else {
            rc = gbfmm_evaluate(ctx, &p, n, d_xyzq, d_out, d_workspace, workspace_bytes, s);
            e = cudaStreamEndCapture(s, &graph);
            if (rc == GBFMM_OK && (e != cudaSuccess || !graph)) rc = cuda_fail(ctx, e, "cudaStreamEndCapture");
        }
    }
    cudaGraphExec_t exec = nullptr;
    // the kernel nodes keep the priorities of the streams they were captured from (the near
    // field's low-priority stream beside the expansions' high-priority one)
    if (rc == GBFMM_OK &&
        (e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority)) != cudaSuccess)
        rc = cuda_fail(ctx, e, "cudaGraphInstantiate");
    cudaStreamDestroy(s);
    if (rc != GBFMM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    gbfmm_graph *g = new (std::nothrow) gbfmm_graph();
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return GBFMM_ENOMEM;
    }
    g->device = ctx->device;
    g->graph = graph;
    g->exec = exec;
    *out = g;
    return GBFMM_OK;
}

int gbfmm_graph_launch(gbfmm_graph *g, void *stream)
{
    if (!g) return GBFMM_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return GBFMM_ECUDA;
    return cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? GBFMM_OK : GBFMM_ECUDA;
}

int gbfmm_graph_destroy(gbfmm_graph *g)
{
    if (!g) return GBFMM_OK;
    cudaSetDevice(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return GBFMM_OK;
}

// times every (leaf size, P2P leaves per CTA) pair: one warm-up and one timed evaluation each
static int tune_impl(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, const int32_t *candidates,
                     int32_t ncand, const int32_t *lpcs, int32_t nlpc, int32_t *best_leaf, int32_t *best_lpc,
                     float *best_ms)
{
    if (!ctx || !prm || !candidates || ncand <= 0 || !best_leaf || n <= 0 || !d_xyzq || nlpc <= 0 || !lpcs)
        return GBFMM_EINVAL;
    for (int32_t j = 0; j < nlpc; ++j)
        if (lpcs[j] < 0 || lpcs[j] > gbfmm::kMaxP2PLeavesPerCta) return GBFMM_EINVAL;
    const int keep = ctx->p2p_leaves_per_cta;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    // output and workspace: the context's host-path buffers, grown to the largest candidate
    size_t ws_max = 0;
    for (int32_t i = 0; i < ncand; ++i) {
        gbfmm_params p = *prm;
        p.leaf_size = candidates[i];
        size_t ws = 0;
        if (gbfmm_plan(&p, n, nullptr, &ws) == GBFMM_OK && ws > ws_max) ws_max = ws;
    }
    if (ctx->h_cap_n < n) {
        cudaFree(ctx->h_in);
        cudaFree(ctx->h_out);
        ctx->h_in = ctx->h_out = nullptr;
        ctx->h_cap_n = 0;
        if ((e = cudaMalloc(&ctx->h_in, 16 * (size_t)n)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(in)");
        if ((e = cudaMalloc(&ctx->h_out, 16 * (size_t)n)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(out)");
        ctx->h_cap_n = n;
    }
    if (ws_max > ctx->h_ws_bytes) {
        cudaFree(ctx->h_ws);
        ctx->h_ws = nullptr;
        ctx->h_ws_bytes = 0;
        if ((e = cudaMalloc(&ctx->h_ws, ws_max)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(workspace)");
        ctx->h_ws_bytes = ws_max;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&t0) != cudaSuccess ||
        cudaEventCreate(&t1) != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        if (t0) cudaEventDestroy(t0);
        return cuda_fail(ctx, cudaGetLastError(), "stream / events");
    }
    int rc = GBFMM_OK, found = 0;
    float best = FLT_MAX;
    for (int32_t k = 0; k < ncand * nlpc && rc == GBFMM_OK; ++k) {
        const int32_t i = k / nlpc, j = k % nlpc;
        gbfmm_params p = *prm;
        p.leaf_size = candidates[i];
        p.flags &= ~GBFMM_FLAG_STAGE_TIMING;
        if (gbfmm_plan(&p, n, nullptr, nullptr) != GBFMM_OK) continue;  // an invalid candidate is skipped
        ctx->p2p_leaves_per_cta = lpcs[j];
        rc = gbfmm_evaluate(ctx, &p, n, d_xyzq, ctx->h_out, ctx->h_ws, ctx->h_ws_bytes, s);  // warm-up
        if (rc != GBFMM_OK) break;
        cudaEventRecord(t0, s);
        rc = gbfmm_evaluate(ctx, &p, n, d_xyzq, ctx->h_out, ctx->h_ws, ctx->h_ws_bytes, s);
        cudaEventRecord(t1, s);
        if (rc != GBFMM_OK) break;
        rc = gbfmm_sync_status(ctx, s);
        float ms = 0.f;
        if (rc == GBFMM_OK && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms < best) {
            best = ms;
            *best_leaf = candidates[i];
            if (best_lpc) *best_lpc = lpcs[j];
            found = 1;
        }
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaStreamDestroy(s);
    ctx->p2p_leaves_per_cta = keep;
    if (rc != GBFMM_OK) return rc;
    if (!found) return fail(ctx, GBFMM_EINVAL, "no valid leaf-size candidate");
    if (best_ms) *best_ms = best;
    return GBFMM_OK;
}

int gbfmm_tune_leaf(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, const int32_t *candidates,
                    int32_t ncand, int32_t *best_leaf, float *best_ms)
{
    if (!ctx) return GBFMM_EINVAL;
    const int32_t cur = ctx->p2p_leaves_per_cta;
    return tune_impl(ctx, prm, n, d_xyzq, candidates, ncand, &cur, 1, best_leaf, nullptr, best_ms);
}

int gbfmm_tune(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, const int32_t *leaf_candidates,
               int32_t n_leaf, const int32_t *lpc_candidates, int32_t n_lpc, int32_t *best_leaf, int32_t *best_lpc,
               float *best_ms)
{
    if (!ctx) return GBFMM_EINVAL;
    int32_t lpc = ctx->p2p_leaves_per_cta;
    const int32_t cur = lpc;
    const int rc = n_lpc > 0 ? tune_impl(ctx, prm, n, d_xyzq, leaf_candidates, n_leaf, lpc_candidates, n_lpc,
                                         best_leaf, &lpc, best_ms)
                             : tune_impl(ctx, prm, n, d_xyzq, leaf_candidates, n_leaf, &cur, 1, best_leaf, &lpc,
                                         best_ms);
    if (rc != GBFMM_OK) return rc;
    ctx->p2p_leaves_per_cta = lpc;  // the context keeps the fastest launch shape
    if (best_lpc) *best_lpc = lpc;
    return GBFMM_OK;
}

int gbfmm_set_p2p_leaves_per_cta(gbfmm_ctx *ctx, int32_t leaves)
{
    if (!ctx || leaves < 0 || leaves > gbfmm::kMaxP2PLeavesPerCta) return GBFMM_EINVAL;
    ctx->p2p_leaves_per_cta = leaves;
    return GBFMM_OK;
}

}  // extern "C"
