// Many independent evaluations as one CUDA graph: the C ABI's gbfmm_batch_* and
// gbfmm_evaluate_batch.
//
// A batch is nb instances of uneven sizes, orders and trees whose particles sit at offsets of
// one device array.  Creation evaluates every instance once with counts read back (this sizes
// the adaptive trees), gives each adaptive instance capacities a margin above those counts,
// evaluates it once more laid out for the capacities (allocating what they need), and captures
// all instances into one graph: the instances are spread over concurrent branches (lanes) by
// particle count, each lane evaluating its instances one after another with every stage on the
// lane's stream.  The adaptive instances in the graph read their counts on the device, so a
// replay evaluates whatever particles the arrays then hold, as long as their trees and lists
// fit the capacities; one that outgrows them skips its remaining work and the status word
// reports ENOMEM.  Each instance has its own tree, lists, expansions and root-box scratch, so
// the lanes share nothing but the operator tables and the status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "context.h"
#include "gbfmm.h"

using gbfmm::AdaptCaps;
using gbfmm::AdaptiveState;
using gbfmm::cuda_fail;
using gbfmm::fail;

namespace {

constexpr int kMaxLanes = 64;
constexpr int kEvaluateBatchLanes = 64;  // gbfmm_evaluate_batch's concurrent branches

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Capacities above the counts of an evaluation.  Another sample of the same distribution and
// count can have twice the cells on a small tree (a cell near the split threshold splits or not:
// 119 against 237 cells for two samples of 3981 Plummer particles at leaf size 256), moves cells
// between levels and may reach a few levels deeper; so the cells and leaves get twice the count
// plus a constant, and every level down to three below the deepest may hold as many cells as
// the whole tree (the per-level launches cover the whole capacity, their CTAs past the level's
// cells idle).  The lists grow with the cells, and by more than the cells on small trees (their
// rows fill as the tree deepens): the V rows are bounded by 189 per cell, the others take their
// entries per cell times the cell capacity, with half again as margin.
AdaptCaps with_margin(const AdaptCaps &c)
{
    auto up = [](int64_t v, int64_t slack) { return v + v / 4 + slack; };
    auto per_cell = [&](int64_t v, int64_t cap_cells) {
        const int64_t prop = c.cells > 0 ? (int64_t)std::ceil(1.5 * (double)v * (double)cap_cells / (double)c.cells) : 0;
        return std::max(up(v, 256), prop) + 256;
    };
    AdaptCaps r = c;
    r.cells = 2 * c.cells + 64;
    r.leaves = 2 * c.leaves + 64;
    r.maxl = std::min(gbfmm::kAdaptiveMaxLevel, c.maxl + 3);
    for (int l = 0; l <= gbfmm::kAdaptiveMaxLevel; ++l) r.level[l] = l <= r.maxl ? r.cells : 0;
    for (int k = 0; k < 4; ++k) r.list[k] = k == 1 ? 189 * r.cells : per_cell(c.list[k], r.cells);
    for (int j = 0; j < 2; ++j) r.chain[j] = per_cell(c.chain[j], r.cells);
    return r;
}

struct Instance {
    gbfmm_params prm{};
    int64_t off = 0, n = 0;
    size_t ws_off = 0;  // uniform: workspace offset
    int state = -1;     // adaptive: index into the batch's states
    int lane = 0;
};

}  // namespace

struct gbfmm_batch {
    int device = 0;
    gbfmm_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<Instance> inst;
    std::vector<std::unique_ptr<AdaptiveState>> states;
    std::vector<AdaptCaps> caps;
    void *ws = nullptr;          // uniform workspaces
    float *scratch = nullptr;    // root-box reduction scratch: kBoxPartials floats per lane
    unsigned *counters = nullptr;  // and one counter per lane
    int lanes = 1;
    const float *x = nullptr;
    float *out = nullptr;

    ~gbfmm_batch()
    {
        cudaSetDevice(device);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto &s : states)
            if (s) gbfmm::free_adaptive(*s);
        cudaFree(ws);
        cudaFree(scratch);
        cudaFree(counters);
    }

    // one instance on stream s: counts read back (caps_mode false) or under its capacities
    int run(const Instance &it, bool caps_mode, cudaStream_t s)
    {
        const float *xi = x + 4 * it.off;
        float *oi = out + 4 * it.off;
        float *part = scratch + (size_t)it.lane * gbfmm::kBoxPartials;
        unsigned *cnt = counters + it.lane;
        if (it.state >= 0) {
            AdaptiveState &A = *states[it.state];
            return gbfmm::evaluate_adaptive_in(ctx, A, caps_mode ? &caps[it.state] : nullptr, &it.prm, it.n, xi, oi,
                                               s, part, cnt);
        }
        size_t wsb = 0;
        gbfmm_plan(&it.prm, it.n, nullptr, &wsb);
        return gbfmm::evaluate_uniform_in(ctx, &it.prm, it.n, xi, oi, static_cast<unsigned char *>(ws) + it.ws_off,
                                          wsb, s, part, cnt);
    }
};

extern "C" {

int gbfmm_batch_create(gbfmm_batch **out, gbfmm_ctx *ctx, int32_t nb, const int64_t *offsets, const gbfmm_params *prm,
                       const float *d_xyzq, float *d_out, int32_t lanes)
{
    if (!out || !ctx) return GBFMM_EINVAL;
    *out = nullptr;
    ctx->err.clear();
    if (nb < 1 || !offsets || !prm || !d_xyzq || !d_out) return fail(ctx, GBFMM_EINVAL, "batch: bad argument");
    if (lanes < 1 || lanes > kMaxLanes) return fail(ctx, GBFMM_EINVAL, "batch: lanes must be in [1, 64]");
    if (reinterpret_cast<uintptr_t>(d_xyzq) % 16 != 0 || reinterpret_cast<uintptr_t>(d_out) % 16 != 0)
        return fail(ctx, GBFMM_EINVAL, "particle arrays must be 16-byte aligned");
    if (offsets[0] < 0) return fail(ctx, GBFMM_EINVAL, "batch: offsets must be ascending from >= 0");
    for (int32_t i = 0; i < nb; ++i)
        if (offsets[i + 1] < offsets[i]) return fail(ctx, GBFMM_EINVAL, "batch: offsets must be ascending from >= 0");
    // the arrays of the batch span [offsets[0], offsets[nb]) particles; input and output apart
    const int64_t span = offsets[nb];
    if (d_out < d_xyzq + 4 * span && d_xyzq < d_out + 4 * span)
        return fail(ctx, GBFMM_EINVAL, "batch: d_out overlaps d_xyzq");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");

    std::unique_ptr<gbfmm_batch> b(new (std::nothrow) gbfmm_batch());
    if (!b) return GBFMM_ENOMEM;
    b->device = ctx->device;
    b->ctx = ctx;
    b->x = d_xyzq;
    b->out = d_out;
    // instances: parameters checked, forced serial and untimed (every stage on the lane's stream)
    size_t ws_total = 0;
    for (int32_t i = 0; i < nb; ++i) {
        Instance it;
        it.prm = prm[i];
        it.prm.flags = (it.prm.flags | GBFMM_FLAG_SERIAL) & ~GBFMM_FLAG_STAGE_TIMING;
        it.off = offsets[i];
        it.n = offsets[i + 1] - offsets[i];
        size_t wsb = 0;
        int rc = gbfmm_plan(&it.prm, it.n, nullptr, &wsb);
        if (rc != GBFMM_OK) return fail(ctx, rc, "batch: instance " + std::to_string(i) + " rejected by gbfmm_plan");
        if (it.prm.tree == GBFMM_TREE_ADAPTIVE) {
            if (it.n > 0 && it.prm.leaf_size > 16384)
                return fail(ctx, GBFMM_EUNSUPPORTED, "batch: adaptive leaf sizes above 16384 cannot be captured");
            it.state = (int)b->states.size();
            b->states.emplace_back(new (std::nothrow) AdaptiveState());
            if (!b->states.back()) return GBFMM_ENOMEM;
        } else {
            it.ws_off = ws_total;
            ws_total += align256(wsb);
        }
        if (it.n > 0) b->inst.push_back(it);
    }
    // lanes: instances by particle count, largest first, each to the lane with the fewest
    // particles so far; within a lane in batch order
    b->lanes = std::max(1, std::min<int>(lanes, (int)b->inst.size()));
    {
        std::vector<int> order(b->inst.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->inst[a].n > b->inst[c].n; });
        std::vector<int64_t> load(b->lanes, 0);
        for (int i : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->inst[i].lane = k;
            load[k] += b->inst[i].n;
        }
    }
    if ((ws_total && cudaMalloc(&b->ws, ws_total) != cudaSuccess) ||
        cudaMalloc(&b->scratch, sizeof(float) * gbfmm::kBoxPartials * b->lanes) != cudaSuccess ||
        cudaMalloc(&b->counters, sizeof(unsigned) * b->lanes) != cudaSuccess ||
        cudaMemset(b->counters, 0, sizeof(unsigned) * b->lanes) != cudaSuccess)
        return fail(ctx, GBFMM_ENOMEM, "batch: workspace allocation");

    cudaStream_t s0 = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaStreamCreate");
    std::vector<cudaStream_t> ls(b->lanes, nullptr);
    std::vector<cudaEvent_t> ev(b->lanes + 1, nullptr);
    auto cleanup = [&]() {
        for (cudaStream_t s : ls)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t v : ev)
            if (v) cudaEventDestroy(v);
        cudaStreamDestroy(s0);
    };
    int rc = GBFMM_OK;
    // 1. counts read back; 2. the adaptive instances once more under their capacities (this
    // allocates what the captured form uses and checks that it runs)
    for (const Instance &it : b->inst)
        if ((rc = b->run(it, false, s0)) != GBFMM_OK) break;
    if (rc == GBFMM_OK) rc = gbfmm_sync_status(ctx, s0);
    if (rc == GBFMM_OK) {
        b->caps.resize(b->states.size());
        for (const Instance &it : b->inst) {
            if (it.state < 0) continue;
            const AdaptCaps &c = b->states[it.state]->counts;
            if (!c.valid) {
                rc = fail(ctx, GBFMM_EUNSUPPORTED, "batch: an adaptive instance cannot be laid out for capture");
                break;
            }
            b->caps[it.state] = with_margin(c);
        }
    }
    if (rc == GBFMM_OK)
        for (const Instance &it : b->inst)
            if (it.state >= 0 && (rc = b->run(it, true, s0)) != GBFMM_OK) break;
    if (rc == GBFMM_OK) rc = gbfmm_sync_status(ctx, s0);
    // 3. capture: lanes forked from s0 and joined back into it
    for (int k = 0; rc == GBFMM_OK && k < b->lanes; ++k)
        if ((e = cudaStreamCreateWithFlags(&ls[k], cudaStreamNonBlocking)) != cudaSuccess)
            rc = cuda_fail(ctx, e, "cudaStreamCreate");
    for (int k = 0; rc == GBFMM_OK && k <= b->lanes; ++k)
        if ((e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming)) != cudaSuccess)
            rc = cuda_fail(ctx, e, "cudaEventCreate");
    if (rc == GBFMM_OK) {
        if ((e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            rc = cuda_fail(ctx, e, "cudaStreamBeginCapture");
        } else {
            cudaEventRecord(ev[b->lanes], s0);
            for (int k = 0; k < b->lanes; ++k) cudaStreamWaitEvent(ls[k], ev[b->lanes], 0);
            for (const Instance &it : b->inst) {
                rc = b->run(it, it.state >= 0, ls[it.lane]);
                if (rc != GBFMM_OK) break;
            }
            for (int k = 0; k < b->lanes; ++k) {
                cudaEventRecord(ev[k], ls[k]);
                cudaStreamWaitEvent(s0, ev[k], 0);
            }
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(s0, &graph);
            if (rc == GBFMM_OK && (e != cudaSuccess || !graph)) rc = cuda_fail(ctx, e, "cudaStreamEndCapture");
            b->graph = graph;
        }
    }
    if (rc == GBFMM_OK && (e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
        rc = cuda_fail(ctx, e, "cudaGraphInstantiate");
    cleanup();
    ctx->have_last = false;  // the context's last evaluation is not an exportable one
    if (rc != GBFMM_OK) return rc;
    *out = b.release();
    return GBFMM_OK;
}

int gbfmm_batch_launch(gbfmm_batch *b, void *stream)
{
    if (!b) return GBFMM_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess) return GBFMM_ECUDA;
    cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(b->ctx, e, "cudaGraphLaunch");
}

int gbfmm_batch_info(const gbfmm_batch *b, int32_t *lanes, int64_t *kernel_nodes)
{
    if (!b) return GBFMM_EINVAL;
    if (lanes) *lanes = b->lanes;
    if (kernel_nodes) {
        size_t nn = 0;
        if (cudaGraphGetNodes(b->graph, nullptr, &nn) != cudaSuccess) return GBFMM_ECUDA;
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn && cudaGraphGetNodes(b->graph, nodes.data(), &nn) != cudaSuccess) return GBFMM_ECUDA;
        int64_t k = 0;
        for (cudaGraphNode_t v : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(v, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
        }
        *kernel_nodes = k;
    }
    return GBFMM_OK;
}

int gbfmm_batch_destroy(gbfmm_batch *b)
{
    if (!b) return GBFMM_OK;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    delete b;
    return GBFMM_OK;
}

}  // extern "C"

extern "C" int gbfmm_evaluate_batch(gbfmm_ctx *ctx, int32_t nb, const int64_t *offsets, const gbfmm_params *prm,
                                    const float *d_xyzq, float *d_out, void *stream)
{
    if (!ctx) return GBFMM_EINVAL;
    if (nb < 1 || !offsets || !prm) return fail(ctx, GBFMM_EINVAL, "batch: bad argument");
    const bool same = ctx->batch && ctx->batch_x == d_xyzq && ctx->batch_out == d_out &&
                      (int32_t)ctx->batch_prm.size() == nb &&
                      std::memcmp(ctx->batch_offsets.data(), offsets, sizeof(int64_t) * (nb + 1)) == 0 &&
                      std::memcmp(ctx->batch_prm.data(), prm, sizeof(gbfmm_params) * nb) == 0;
    if (!same) {
        gbfmm_batch_destroy(ctx->batch);
        ctx->batch = nullptr;
        ctx->batch_prm.clear();
        const int rc = gbfmm_batch_create(&ctx->batch, ctx, nb, offsets, prm, d_xyzq, d_out, kEvaluateBatchLanes);
        if (rc != GBFMM_OK) return rc;
        ctx->batch_offsets.assign(offsets, offsets + nb + 1);
        ctx->batch_prm.assign(prm, prm + nb);
        ctx->batch_x = d_xyzq;
        ctx->batch_out = d_out;
    }
    return gbfmm_batch_launch(ctx->batch, stream);
}
