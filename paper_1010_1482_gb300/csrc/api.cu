// C ABI of libgbfmm (declared in include/gbfmm.h): context, planning, the evaluation
// pipeline (tree front end -> upward pass -> M2L or M2P -> downward pass -> P2P) and the
// debug exports.  Host code here only sizes buffers and enqueues kernels; no arithmetic of
// the method runs on the host.
#include "common.cuh"
#include "gbfmm.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

namespace gbfmm {
void init_expansion_constants();
void init_m2l_constants();
void init_m2l_f16_constants();
void init_m2l_rot_constants();
}  // namespace gbfmm

using namespace gbfmm;

namespace gbfmm {
static thread_local int64_t tl_launches = 0;
void note_launches(int k) { tl_launches += k; }
int64_t launch_count() { return tl_launches; }

int sm_count()
{
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 0;
    }();
    return n;
}
}  // namespace gbfmm

#include "context.h"

int gbfmm::order_slot(int p)
{
    for (int i = 0; i < 4; ++i)
        if (kOrders[i] == p) return i;
    return -1;
}

int gbfmm::fail(gbfmm_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int gbfmm::cuda_fail(gbfmm_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, GBFMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

int uniform_depth(int64_t n, int64_t leaf)
{
    int L = 0;
    while (n > leaf * (int64_t(1) << (3 * L))) {
        ++L;
        if (L > 20) break;
    }
    return L;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int check_params(const gbfmm_params *prm, int64_t n, int *L_out, std::string *msg)
{
    if (!prm) {
        *msg = "params is NULL";
        return GBFMM_EINVAL;
    }
    if (n < 0) {
        *msg = "n < 0";
        return GBFMM_EINVAL;
    }
    if (order_slot(prm->p) < 0) {
        *msg = "order p not compiled (4, 6, 8, 10)";
        return GBFMM_EUNSUPPORTED;
    }
    if (prm->leaf_size < 1) {
        *msg = "leaf_size < 1";
        return GBFMM_EINVAL;
    }
    if (prm->tree != GBFMM_TREE_UNIFORM && prm->tree != GBFMM_TREE_ADAPTIVE) {
        *msg = "unknown tree";
        return GBFMM_EINVAL;
    }
    if (prm->method != GBFMM_METHOD_FMM && prm->method != GBFMM_METHOD_TREECODE) {
        *msg = "unknown method";
        return GBFMM_EINVAL;
    }
    if (!(prm->eps2 >= 0.0) || !isfinite(prm->eps2)) {
        *msg = "eps2 must be finite and >= 0";
        return GBFMM_EINVAL;
    }
    if (prm->has_box) {
        if (!(prm->box_side > 0.0) || !isfinite(prm->box_side) || !isfinite(prm->box_origin[0]) ||
            !isfinite(prm->box_origin[1]) || !isfinite(prm->box_origin[2])) {
            *msg = "box must be finite with side > 0";
            return GBFMM_EINVAL;
        }
    }
    if (n > (int64_t)0x7fffffff) {
        *msg = "n exceeds 2^31 - 1";
        return GBFMM_EUNSUPPORTED;
    }
    if (prm->tree == GBFMM_TREE_ADAPTIVE) {
        *L_out = kAdaptiveMaxLevel;
        return GBFMM_OK;
    }
    int L = uniform_depth(n, prm->leaf_size);
    if (L > kMaxLevel) {
        *msg = "tree depth exceeds 10 (raise leaf_size)";
        return GBFMM_EUNSUPPORTED;
    }
    *L_out = L;
    return GBFMM_OK;
}

Layout make_layout(int64_t n, int L, int P)
{
    Layout lo{};
    lo.n = n;
    lo.L = L;
    lo.P = P;
    lo.ncells = level_offset(L + 1);
    lo.nleaves = int64_t(1) << (3 * L);
    lo.rs_blocks = (n + 4095) / 4096;
    const int64_t C = lo.ncells, NL = lo.nleaves;
    const int64_t C2 = L >= 2 ? C - level_offset(2) : 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    lo.box = take(sizeof(Box));
    lo.keys0 = take(4 * (size_t)n);
    lo.keys1 = take(4 * (size_t)n);
    lo.idx0 = take(4 * (size_t)n);
    lo.idx1 = take(4 * (size_t)n);
    lo.sx = take(16 * (size_t)n);
    lo.far = take(32 * (size_t)n);  // far field (16 B), or the near-field sums (32 B)
    lo.rs_hist = take(sort_scratch_bytes(n, 3 * L));
    size_t tmpw = std::max({exclusive_scan_tmp_words(256 * lo.rs_blocks), exclusive_scan_tmp_words(C),
                            exclusive_scan_tmp_words(NL)});
    lo.scan_tmp = take(4 * tmpw);
    lo.cell_begin = take(4 * (size_t)C);
    lo.cell_end = take(4 * (size_t)C);
    lo.p2p_len = take(4 * (size_t)NL);
    lo.p2p_offs = take(4 * (size_t)(NL + 1));
    lo.p2p_ids = take(4 * (size_t)(27 * NL));
    lo.m2l_len = take(4 * (size_t)C);
    lo.m2l_offs = take(4 * (size_t)(C + 1));
    lo.m2l_ids = take(4 * (size_t)(189 * C2 + 1));
    lo.m2l_code = take(2 * (size_t)(189 * C2 + 1));
    lo.M = take(4 * (size_t)C * P * P);
    lo.Lc = take(4 * (size_t)C * P * P);
    lo.cscale = take(std::max((size_t)C, m2l_blk_scale_bytes(L)));
    lo.geo = take(4 * geo_floats(L));
    lo.presplit = take(std::max(presplit_bytes(P, C), m2l_blk_presplit_bytes(P, L)));
    lo.lpart = take(m2l_blk_part_bytes(P, L));
    lo.total = off;
    return lo;
}

template <class T>
T *at(void *base, size_t off)
{
    return reinterpret_cast<T *>(static_cast<unsigned char *>(base) + off);
}

}  // namespace

int gbfmm::ensure_ops(gbfmm_ctx *ctx, int P, cudaStream_t s, bool *built_now)
{
    OpsCache &c = ctx->ops[order_slot(P)];
    *built_now = false;
    if (c.built) return GBFMM_OK;
    const size_t PR = ((size_t)P * P + 7) / 8 * 8;
    cudaError_t e;
    if ((e = cudaMalloc(&c.m2l, kM2LCodes * (size_t)P * P * PR * sizeof(float))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(m2l ops)");
    if ((e = cudaMalloc(&c.m2m, 8 * (size_t)P * P * PR * sizeof(float))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(m2m ops)");
    if ((e = cudaMalloc(&c.l2l, 8 * (size_t)P * P * PR * sizeof(float))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(l2l ops)");
    launch_build_operators(P, c.m2l, c.m2m, c.l2l, s);
    if ((e = cudaMalloc(&c.m2l_f16, m2l_f16_table_bytes(P))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(m2l FP16 tensor-core ops)");
    launch_build_m2l_f16(P, c.m2l, c.m2l_f16, s);
    c.P = P;
    c.built = true;
    *built_now = true;
    return GBFMM_OK;
}

// the rotation factors of the M2L operators: computed on the host in FP64 and checked against
// the dense operators at first use of order P (synchronous)
static int ensure_rot(gbfmm_ctx *ctx, int P)
{
    OpsCache &c = ctx->ops[order_slot(P)];
    if (c.m2l_rot) return GBFMM_OK;
    cudaError_t e = cudaMalloc(&c.m2l_rot, m2l_rot_table_bytes(P));
    if (e != cudaSuccess) {
        c.m2l_rot = nullptr;
        return cuda_fail(ctx, e, "cudaMalloc(m2l rotation factors)");
    }
    const int rc = build_m2l_rot(P, c.m2l_rot);
    if (rc != 0) {
        cudaFree(c.m2l_rot);
        c.m2l_rot = nullptr;
        return fail(ctx, GBFMM_ECUDA, "rotation factors of the M2L operators failed their check (" + std::to_string(rc) + ")");
    }
    return GBFMM_OK;
}

// the block operators of the uniform tree's M2L (built on the stream at first use of order P)
int gbfmm::ensure_blk(gbfmm_ctx *ctx, int P, cudaStream_t s)
{
    OpsCache &c = ctx->ops[order_slot(P)];
    if (c.m2l_blk) return GBFMM_OK;
    cudaError_t e = cudaMalloc(&c.m2l_blk, m2l_blk_table_bytes(P));
    if (e != cudaSuccess) {
        c.m2l_blk = nullptr;
        return cuda_fail(ctx, e, "cudaMalloc(m2l block operators)");
    }
    launch_build_m2l_blk(P, c.m2l, c.m2l_blk, s);
    return GBFMM_OK;
}

extern "C" {

int gbfmm_version(void) { return GBFMM_VERSION; }

int gbfmm_default_params(gbfmm_params *prm)
{
    if (!prm) return GBFMM_EINVAL;
    memset(prm, 0, sizeof(*prm));
    prm->p = 10;
    prm->leaf_size = 64;
    prm->tree = GBFMM_TREE_UNIFORM;
    prm->method = GBFMM_METHOD_FMM;
    prm->eps2 = 0.0;
    prm->has_box = 0;
    prm->box_side = 1.0;
    return GBFMM_OK;
}

int gbfmm_create(gbfmm_ctx **out, int device)
{
    if (!out) return GBFMM_EINVAL;
    *out = nullptr;
    gbfmm_ctx *ctx = new (std::nothrow) gbfmm_ctx();
    if (!ctx) return GBFMM_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return GBFMM_ECUDA;
    }
    bool ok = cudaMalloc(&ctx->d_status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&ctx->d_counter, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&ctx->d_partials, kBoxPartials * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&ctx->d_zero, 128 * sizeof(float)) == cudaSuccess;
    if (ok)
        ok = cudaMemset(ctx->d_status, 0, sizeof(int)) == cudaSuccess &&
             cudaMemset(ctx->d_counter, 0, sizeof(unsigned)) == cudaSuccess &&
             cudaMemset(ctx->d_zero, 0, 128 * sizeof(float)) == cudaSuccess;
    for (int i = 0; ok && i <= kStages; ++i) ok = cudaEventCreate(&ctx->ev[i]) == cudaSuccess;
    for (int i = 0; ok && i < 3; ++i) ok = cudaEventCreate(&ctx->ev_aux[i]) == cudaSuccess;
    if (ok) {
        int least = 0, greatest = 0;
        ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
             cudaStreamCreateWithPriority(&ctx->s_far, cudaStreamNonBlocking, greatest) == cudaSuccess &&
             cudaStreamCreateWithPriority(&ctx->s_near, cudaStreamNonBlocking, least) == cudaSuccess;
        for (cudaEvent_t *e : {&ctx->ev_fork, &ctx->ev_near, &ctx->ev_join})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok) {
        init_expansion_constants();
        init_m2l_constants();
        init_m2l_f16_constants();
        init_m2l_rot_constants();
        ok = cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        gbfmm_destroy(ctx);
        return GBFMM_ECUDA;
    }
    *out = ctx;
    return GBFMM_OK;
}

int gbfmm_destroy(gbfmm_ctx *ctx)
{
    if (!ctx) return GBFMM_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    gbfmm_batch_destroy(ctx->batch);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_counter);
    cudaFree(ctx->d_partials);
    cudaFree(ctx->d_zero);
    for (auto &c : ctx->ops) {
        cudaFree(c.m2l);
        cudaFree(c.m2m);
        cudaFree(c.l2l);
        cudaFree(c.m2l_f16);
        cudaFree(c.m2l_blk);
        cudaFree(c.m2l_rot);
    }
    cudaFree(ctx->h_in);
    cudaFree(ctx->h_out);
    cudaFree(ctx->h_ws);
    free_adaptive(ctx->ad);
    for (int i = 0; i <= kStages; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_near, ctx->ev_join, ctx->ev_aux[0], ctx->ev_aux[1], ctx->ev_aux[2]})
        if (e) cudaEventDestroy(e);
    if (ctx->s_far) cudaStreamDestroy(ctx->s_far);
    if (ctx->s_near) cudaStreamDestroy(ctx->s_near);
    delete ctx;
    return GBFMM_OK;
}

const char *gbfmm_last_error(const gbfmm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gbfmm_plan(const gbfmm_params *prm, int64_t n, int32_t *levels, size_t *workspace_bytes)
{
    std::string msg;
    int L = 0;
    int rc = check_params(prm, n, &L, &msg);
    if (rc != GBFMM_OK) return rc;
    if (levels) *levels = L;
    if (prm->tree == GBFMM_TREE_ADAPTIVE) {
        if (workspace_bytes) *workspace_bytes = 0;
        return GBFMM_OK;
    }
    Layout lo = make_layout(n, L, prm->p);
    if (workspace_bytes) *workspace_bytes = lo.total;
    return GBFMM_OK;
}

int gbfmm_evaluate(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                   void *d_workspace, size_t workspace_bytes, void *stream)
{
    if (!ctx) return GBFMM_EINVAL;
    ctx->err.clear();
    std::string msg;
    int L = 0;
    int rc = check_params(prm, n, &L, &msg);
    if (rc != GBFMM_OK) return fail(ctx, rc, msg);
    if (n == 0) return GBFMM_OK;
    if (prm->tree == GBFMM_TREE_ADAPTIVE) {
        if (!d_xyzq || !d_out) return fail(ctx, GBFMM_EINVAL, "null device pointer");
        if (reinterpret_cast<uintptr_t>(d_xyzq) % 16 != 0 || reinterpret_cast<uintptr_t>(d_out) % 16 != 0)
            return fail(ctx, GBFMM_EINVAL, "particle arrays must be 16-byte aligned");
        if (d_xyzq == d_out) return fail(ctx, GBFMM_EINVAL, "d_out aliases d_xyzq");
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
        ctx->have_last = false;
        const int64_t launches0 = tl_launches;
        rc = evaluate_adaptive(ctx, prm, n, d_xyzq, d_out, static_cast<cudaStream_t>(stream));
        ctx->launches_last = tl_launches - launches0;
        if (rc != GBFMM_OK) return rc;
        ctx->have_last = true;
        ctx->last_adaptive = true;
        ctx->last_method = prm->method;
        ctx->timed_last = (prm->flags & GBFMM_FLAG_STAGE_TIMING) != 0;
        return GBFMM_OK;
    }
    return evaluate_uniform_in(ctx, prm, n, d_xyzq, d_out, d_workspace, workspace_bytes,
                               static_cast<cudaStream_t>(stream), ctx->d_partials, ctx->d_counter);
}

}  // extern "C"

namespace gbfmm {

int evaluate_uniform_in(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                        void *d_workspace, size_t workspace_bytes, cudaStream_t stream, float *partials,
                        unsigned *counter)
{
    set_p2p_leaves_per_cta(ctx->p2p_leaves_per_cta);
    std::string msg;
    int L = 0;
    int rc = check_params(prm, n, &L, &msg);
    if (rc != GBFMM_OK) return fail(ctx, rc, msg);
    if (n == 0) return GBFMM_OK;
    if (!d_xyzq || !d_out || !d_workspace) return fail(ctx, GBFMM_EINVAL, "null device pointer");
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return fail(ctx, GBFMM_EINVAL, "workspace not 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_xyzq) % 16 != 0 || reinterpret_cast<uintptr_t>(d_out) % 16 != 0)
        return fail(ctx, GBFMM_EINVAL, "particle arrays must be 16-byte aligned");
    if (d_xyzq == d_out) return fail(ctx, GBFMM_EINVAL, "d_out aliases d_xyzq");
    const int P = prm->p;
    Layout lo = make_layout(n, L, P);
    if (workspace_bytes < lo.total) return fail(ctx, GBFMM_ENOMEM, "workspace smaller than gbfmm_plan's size");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool timing = (prm->flags & GBFMM_FLAG_STAGE_TIMING) != 0;
    auto mark = [&](int k) {
        if (timing) cudaEventRecord(ctx->ev[k], s);
    };

    void *ws = d_workspace;
    const float4 *x = reinterpret_cast<const float4 *>(d_xyzq);
    float4 *out = reinterpret_cast<float4 *>(d_out);
    Box *box = at<Box>(ws, lo.box);
    uint32_t *k0 = at<uint32_t>(ws, lo.keys0), *k1 = at<uint32_t>(ws, lo.keys1);
    uint32_t *v0 = at<uint32_t>(ws, lo.idx0), *v1 = at<uint32_t>(ws, lo.idx1);
    float4 *sx = at<float4>(ws, lo.sx), *far = at<float4>(ws, lo.far);
    uint32_t *hist = at<uint32_t>(ws, lo.rs_hist), *scan_tmp = at<uint32_t>(ws, lo.scan_tmp);
    int32_t *begin = at<int32_t>(ws, lo.cell_begin), *end = at<int32_t>(ws, lo.cell_end);
    uint32_t *p2p_len = at<uint32_t>(ws, lo.p2p_len), *p2p_offs = at<uint32_t>(ws, lo.p2p_offs);
    int32_t *p2p_ids = at<int32_t>(ws, lo.p2p_ids);
    uint32_t *m2l_len = at<uint32_t>(ws, lo.m2l_len), *m2l_offs = at<uint32_t>(ws, lo.m2l_offs);
    int32_t *m2l_ids = at<int32_t>(ws, lo.m2l_ids);
    uint16_t *m2l_code = at<uint16_t>(ws, lo.m2l_code);
    float *M = at<float>(ws, lo.M), *Lc = at<float>(ws, lo.Lc);
    float *geo = at<float>(ws, lo.geo);

    // operator tables (once per order and context)
    bool built_now = false;
    if (L >= 2) {
        if (timing) cudaEventRecord(ctx->ev[kStages], s);
        rc = ensure_ops(ctx, P, s, &built_now);
        if (rc != GBFMM_OK) return rc;
    }
    const OpsCache &ops = ctx->ops[order_slot(P)];

    const int64_t launches0 = tl_launches;
    mark(0);
    launch_bbox(x, n, prm->has_box, prm->box_origin, prm->box_side, box, partials, counter, ctx->d_status, s);
    launch_keys(x, n, box, L, k0, v0, s);
    if (L >= 2) launch_geo_levels(box, L, geo, s);
    mark(1);
    uint32_t *skeys = nullptr, *perm = nullptr;
    launch_sort_gather(k0, k1, v0, v1, n, 3 * L, hist, ctx->d_status, x, sx, &skeys, &perm, s);
    mark(2);
    launch_cells(skeys, n, L, begin, end, s);
    // the block M2L reads no M2L list: then only the P2P rows are built, on the near field's
    // stream (the M2L rows are built on demand by gbfmm_export_lists)
    const bool cores = (prm->flags & GBFMM_FLAG_M2L_CUDA_CORES) != 0;
    const bool gathered = (prm->flags & GBFMM_FLAG_M2L_GATHERED) != 0;
    const bool rot = (prm->flags & GBFMM_FLAG_M2L_ROTATION) != 0;
    const bool blk = L >= 2 && prm->method == GBFMM_METHOD_FMM && !cores && !gathered && !rot;
    auto p2p_lists = [&](cudaStream_t st) {
        launch_p2p_list_count(L, begin, end, p2p_len, st);
        launch_exclusive_scan(p2p_len, p2p_offs, lo.nleaves, scan_tmp, st);
        launch_p2p_list_fill(L, begin, end, p2p_offs, p2p_ids, st);
    };
    if (!blk) {
        launch_list_count(L, begin, end, p2p_len, m2l_len, s);
        launch_exclusive_scan(p2p_len, p2p_offs, lo.nleaves, scan_tmp, s);
        launch_exclusive_scan(m2l_len, m2l_offs, lo.ncells, scan_tmp, s);
        launch_list_fill(L, begin, end, p2p_offs, p2p_ids, m2l_offs, m2l_ids, m2l_code, s);
    }
    mark(3);
    // near field beside the far field (FMM): P2P writes its compensated sums, L2P adds the far
    // field to them and writes the output; concurrently on the context's two streams unless the
    // evaluation is timed or serial
    const bool split = L >= 2 && prm->method == GBFMM_METHOD_FMM && p2p_near_supported();
    const bool fork = split && (prm->flags & GBFMM_FLAG_SERIAL) == 0;
    float4 *near = split ? far : nullptr;
    const cudaStream_t s_main = s;
    if (fork) {
        cudaEventRecord(ctx->ev_fork, s_main);
        cudaStreamWaitEvent(ctx->s_far, ctx->ev_fork, 0);
        cudaStreamWaitEvent(ctx->s_near, ctx->ev_fork, 0);
        s = ctx->s_far;
        if (timing) cudaEventRecord(ctx->ev_aux[0], ctx->s_near);
        if (blk) p2p_lists(ctx->s_near);
        launch_p2p_near(L, n, sx, begin, end, p2p_offs, p2p_ids, (float)prm->eps2, near, ctx->d_status, ctx->s_near);
        if (timing) cudaEventRecord(ctx->ev_aux[1], ctx->s_near);
        cudaEventRecord(ctx->ev_near, ctx->s_near);
    }
    if (blk && !fork) p2p_lists(s);  // serial: the P2P rows now, P2P after the far field
    if (L >= 2) launch_p2m(P, L, geo, sx, begin, end, M, s);
    mark(4);
    if (L >= 2)
        for (int l = L - 1; l >= 2; --l) launch_m2m(P, l, begin, end, ops.m2m, M, s);
    mark(5);
    if (L >= 2) {
        if (blk) {
            rc = ensure_blk(ctx, P, s);
            if (rc != GBFMM_OK) return rc;
            int8_t *pscale = at<int8_t>(ws, lo.cscale);
            void *ps = at<void>(ws, lo.presplit);
            launch_blk_presplit(P, L, begin, end, M, ps, pscale, s);
            if (launch_m2l_blk(P, L, begin, end, ps, pscale, ops.m2l_blk, Lc, at<float>(ws, lo.lpart), ctx->d_status,
                               s, fork ? sm_count() : 0) != 0)
                return fail(ctx, GBFMM_ECUDA, "TMA tensor map encoding failed");
        } else if (prm->method == GBFMM_METHOD_FMM && rot && !cores) {
            rc = ensure_rot(ctx, P);
            if (rc != GBFMM_OK) return rc;
            launch_m2l_rot(P, L, begin, end, m2l_offs, m2l_ids, m2l_code, ops.m2l_rot, M, Lc, s);
        } else if (prm->method == GBFMM_METHOD_FMM && !cores) {
            int8_t *cscale = at<int8_t>(ws, lo.cscale);
            void *ps = at<void>(ws, lo.presplit);
            launch_presplit(P, M, lo.ncells, cscale, ps, s);  // sources split once per cell
            launch_m2l_f16(P, L, begin, end, m2l_offs, m2l_ids, m2l_code, ops.m2l_f16, M, cscale, ps, Lc,
                           ctx->d_status, s, fork ? sm_count() : 0);
        } else if (prm->method == GBFMM_METHOD_FMM)
            launch_m2l(P, L, begin, end, m2l_offs, m2l_ids, m2l_code, ops.m2l, M, Lc, ctx->d_zero, ctx->d_status, s);
        else
            launch_m2p(P, L, geo, sx, begin, end, m2l_offs, m2l_ids, M, far, s);
    }
    mark(6);
    if (L >= 2 && prm->method == GBFMM_METHOD_FMM)
        for (int l = 3; l <= L; ++l) launch_l2l(P, l, begin, end, ops.l2l, Lc, s);
    mark(7);
    if (split) {
        if (fork) {
            mark(8);
            cudaStreamWaitEvent(s, ctx->ev_near, 0);
            if (timing) cudaEventRecord(ctx->ev_aux[2], s);
        } else {
            launch_p2p_near(L, n, sx, begin, end, p2p_offs, p2p_ids, (float)prm->eps2, near, ctx->d_status, s);
            mark(8);
        }
        launch_l2p(P, L, geo, n, sx, skeys, Lc, far, s, near, perm, out);
        mark(9);
        if (fork) {
            cudaEventRecord(ctx->ev_join, s);
            cudaStreamWaitEvent(s_main, ctx->ev_join, 0);
            s = s_main;
        }
    } else {
        if (L >= 2 && prm->method == GBFMM_METHOD_FMM) launch_l2p(P, L, geo, n, sx, skeys, Lc, far, s);
        mark(8);
        launch_p2p(L, n, sx, begin, end, p2p_offs, p2p_ids, L >= 2 ? far : nullptr, perm, (float)prm->eps2, out,
                   ctx->d_status, s);
        mark(9);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");

    ctx->launches_last = tl_launches - launches0;
    ctx->have_last = true;
    ctx->last_adaptive = false;
    ctx->last = lo;
    ctx->last_ws = static_cast<unsigned char *>(ws);
    ctx->last_keys = (size_t)(reinterpret_cast<unsigned char *>(skeys) - ctx->last_ws);
    ctx->last_idx = (size_t)(reinterpret_cast<unsigned char *>(perm) - ctx->last_ws);
    ctx->last_method = prm->method;
    ctx->last_m2l_lists = !blk;
    ctx->timed_last = timing;
    ctx->stage_order_last = fork ? 2 : (split ? 1 : 0);
    ctx->ops_built_last = built_now;
    return GBFMM_OK;
}

}  // namespace gbfmm

extern "C" {

int gbfmm_sync_status(gbfmm_ctx *ctx, void *stream)
{
    if (!ctx) return GBFMM_EINVAL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int st = 0;
    e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status readback");
    cudaMemset(ctx->d_status, 0, sizeof(int));
    if (st & kStatusTimeout) return fail(ctx, GBFMM_ETIMEOUT, "a bounded device wait gave up");
    if (st & kStatusNonFinite) return fail(ctx, GBFMM_EINVAL, "non-finite particle coordinate");
    if (st & kStatusCapacity)
        return fail(ctx, GBFMM_ENOMEM, "an adaptive tree outgrew the capacities of a captured batch (re-create it)");
    return GBFMM_OK;
}

int gbfmm_evaluate_host(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *h_xyzq, float *h_out,
                        void *stream)
{
    if (!ctx) return GBFMM_EINVAL;
    if (n > 0 && (!h_xyzq || !h_out)) return fail(ctx, GBFMM_EINVAL, "null host pointer");
    int32_t L = 0;
    size_t ws = 0;
    int rc = gbfmm_plan(prm, n, &L, &ws);
    if (rc != GBFMM_OK) return fail(ctx, rc, "invalid parameters");
    if (n == 0) return GBFMM_OK;
    cudaSetDevice(ctx->device);
    cudaError_t e;
    if (ctx->h_cap_n < n) {
        cudaFree(ctx->h_in);
        cudaFree(ctx->h_out);
        ctx->h_in = ctx->h_out = nullptr;
        ctx->h_cap_n = 0;
        if ((e = cudaMalloc(&ctx->h_in, 16 * (size_t)n)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(in)");
        if ((e = cudaMalloc(&ctx->h_out, 16 * (size_t)n)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(out)");
        ctx->h_cap_n = n;
    }
    if (ws > 0 && ctx->h_ws_bytes < ws) {
        cudaFree(ctx->h_ws);
        ctx->h_ws = nullptr;
        ctx->h_ws_bytes = 0;
        if ((e = cudaMalloc(&ctx->h_ws, ws)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(workspace)");
        ctx->h_ws_bytes = ws;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpyAsync(ctx->h_in, h_xyzq, 16 * (size_t)n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy in");
    rc = gbfmm_evaluate(ctx, prm, n, ctx->h_in, ctx->h_out, ctx->h_ws, ctx->h_ws_bytes, stream);
    if (rc != GBFMM_OK) return rc;
    if ((e = cudaMemcpyAsync(h_out, ctx->h_out, 16 * (size_t)n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy out");
    return gbfmm_sync_status(ctx, stream);
}

int gbfmm_direct(gbfmm_ctx *ctx, int64_t n_src, const float *d_src, int64_t n_tgt, const float *d_tgt, double eps2,
                 float *d_out, void *stream)
{
    if (!ctx) return GBFMM_EINVAL;
    if (n_src < 0 || n_tgt < 0) return fail(ctx, GBFMM_EINVAL, "negative size");
    if (!(eps2 >= 0.0)) return fail(ctx, GBFMM_EINVAL, "eps2 must be >= 0");
    if (n_tgt == 0) return GBFMM_OK;
    if ((n_src > 0 && !d_src) || !d_tgt || !d_out) return fail(ctx, GBFMM_EINVAL, "null device pointer");
    cudaSetDevice(ctx->device);
    const int64_t launches0 = tl_launches;
    launch_direct(n_src, reinterpret_cast<const float4 *>(d_src), n_tgt, reinterpret_cast<const float4 *>(d_tgt),
                  (float)eps2, reinterpret_cast<float4 *>(d_out), static_cast<cudaStream_t>(stream));
    ctx->launches_last = tl_launches - launches0;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "direct launch");
}

int gbfmm_export_tree(gbfmm_ctx *ctx, double *origin_side, uint32_t *sorted_leaf_keys, uint32_t *perm,
                      int32_t *begin, int32_t *count)
{
    if (!ctx) return GBFMM_EINVAL;
    if (!ctx->have_last) return fail(ctx, GBFMM_EINVAL, "no evaluation to export");
    if (ctx->last_adaptive) return fail(ctx, GBFMM_EINVAL, "last evaluation used the adaptive tree");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    const Layout &lo = ctx->last;
    if (origin_side) {
        Box b;
        cudaMemcpy(&b, ctx->last_ws + lo.box, sizeof(Box), cudaMemcpyDeviceToHost);
        origin_side[0] = b.origin[0];
        origin_side[1] = b.origin[1];
        origin_side[2] = b.origin[2];
        origin_side[3] = b.side;
    }
    if (sorted_leaf_keys) cudaMemcpy(sorted_leaf_keys, ctx->last_ws + ctx->last_keys, 4 * lo.n, cudaMemcpyDeviceToHost);
    if (perm) cudaMemcpy(perm, ctx->last_ws + ctx->last_idx, 4 * lo.n, cudaMemcpyDeviceToHost);
    if (begin || count) {
        std::vector<int32_t> b(lo.ncells), en(lo.ncells);
        cudaMemcpy(b.data(), ctx->last_ws + lo.cell_begin, 4 * lo.ncells, cudaMemcpyDeviceToHost);
        cudaMemcpy(en.data(), ctx->last_ws + lo.cell_end, 4 * lo.ncells, cudaMemcpyDeviceToHost);
        for (int64_t g = 0; g < lo.ncells; ++g) {
            int32_t c = en[g] - b[g];
            if (begin) begin[g] = c > 0 ? b[g] : 0;
            if (count) count[g] = c;
        }
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "export copy");
}

int gbfmm_export_lists(gbfmm_ctx *ctx, int kind, int32_t *offs, int32_t *ids, int64_t cap, int64_t *n_entries)
{
    if (!ctx) return GBFMM_EINVAL;
    if (!ctx->have_last) return fail(ctx, GBFMM_EINVAL, "no evaluation to export");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    if (ctx->last_adaptive) {
        if (kind < GBFMM_LIST_U || kind > GBFMM_LIST_X)
            return fail(ctx, GBFMM_EINVAL, "list kind does not match the adaptive tree");
        return export_adaptive_list(ctx, kind - GBFMM_LIST_U, offs, ids, cap, n_entries);
    }
    if (kind != GBFMM_LIST_P2P && kind != GBFMM_LIST_M2L) return fail(ctx, GBFMM_EINVAL, "unknown list kind");
    const Layout &lo = ctx->last;
    if (kind == GBFMM_LIST_M2L && !ctx->last_m2l_lists && lo.L >= 2) {
        // the evaluation's block M2L read no list: build the rows now from its cells
        unsigned char *w = ctx->last_ws;
        const int32_t *cb = reinterpret_cast<const int32_t *>(w + lo.cell_begin);
        const int32_t *ce = reinterpret_cast<const int32_t *>(w + lo.cell_end);
        uint32_t *p2p_len = reinterpret_cast<uint32_t *>(w + lo.p2p_len), *p2p_offs = reinterpret_cast<uint32_t *>(w + lo.p2p_offs);
        uint32_t *m2l_len = reinterpret_cast<uint32_t *>(w + lo.m2l_len), *m2l_offs = reinterpret_cast<uint32_t *>(w + lo.m2l_offs);
        uint32_t *tmp = reinterpret_cast<uint32_t *>(w + lo.scan_tmp);
        launch_list_count(lo.L, cb, ce, p2p_len, m2l_len, 0);
        launch_exclusive_scan(p2p_len, p2p_offs, lo.nleaves, tmp, 0);
        launch_exclusive_scan(m2l_len, m2l_offs, lo.ncells, tmp, 0);
        launch_list_fill(lo.L, cb, ce, p2p_offs, reinterpret_cast<int32_t *>(w + lo.p2p_ids), m2l_offs,
                         reinterpret_cast<int32_t *>(w + lo.m2l_ids), reinterpret_cast<uint16_t *>(w + lo.m2l_code), 0);
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "M2L list build");
        ctx->last_m2l_lists = true;
    }
    const int64_t rows = kind == GBFMM_LIST_P2P ? lo.nleaves : lo.ncells;
    std::vector<uint32_t> o(rows + 1);
    cudaMemcpy(o.data(), ctx->last_ws + (kind == GBFMM_LIST_P2P ? lo.p2p_offs : lo.m2l_offs), 4 * (rows + 1),
               cudaMemcpyDeviceToHost);
    const int64_t ne = o[rows];
    if (n_entries) *n_entries = ne;
    if (offs)
        for (int64_t r = 0; r <= rows; ++r) offs[r] = (int32_t)o[r];
    if (ids) {
        if (cap < ne) return fail(ctx, GBFMM_ENOMEM, "ids capacity too small");
        cudaMemcpy(ids, ctx->last_ws + (kind == GBFMM_LIST_P2P ? lo.p2p_ids : lo.m2l_ids), 4 * ne,
                   cudaMemcpyDeviceToHost);
        for (int64_t r = 0; r < rows; ++r) std::sort(ids + o[r], ids + o[r + 1]);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "export copy");
}

int gbfmm_export_expansions(gbfmm_ctx *ctx, int which, double *coef)
{
    if (!ctx || !coef) return GBFMM_EINVAL;
    if (!ctx->have_last) return fail(ctx, GBFMM_EINVAL, "no evaluation to export");
    if (which != 0 && which != 1) return fail(ctx, GBFMM_EINVAL, "which must be 0 (M) or 1 (L)");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    if (ctx->last_adaptive) return export_adaptive_expansions(ctx, which, coef);
    const Layout &lo = ctx->last;
    const int P = lo.P, PP = P * P, NT = P * (P + 1) / 2;
    std::vector<float> v((size_t)lo.ncells * PP);
    std::vector<int32_t> b(lo.ncells), en(lo.ncells);
    Box box;
    cudaMemcpy(&box, ctx->last_ws + lo.box, sizeof(Box), cudaMemcpyDeviceToHost);
    cudaMemcpy(v.data(), ctx->last_ws + (which == 0 ? lo.M : lo.Lc), 4 * v.size(), cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), ctx->last_ws + lo.cell_begin, 4 * lo.ncells, cudaMemcpyDeviceToHost);
    cudaMemcpy(en.data(), ctx->last_ws + lo.cell_end, 4 * lo.ncells, cudaMemcpyDeviceToHost);
    for (int l = 0; l <= lo.L; ++l) {
        const double h = box.side / (double)(int64_t(1) << l);
        const bool formed = lo.L >= 2 && l >= 2 && (which == 0 || ctx->last_method == GBFMM_METHOD_FMM);
        for (int64_t g = level_offset(l); g < level_offset(l + 1); ++g) {
            double *c = coef + (size_t)g * 2 * NT;
            const bool ok = formed && en[g] > b[g];
            for (int n = 0; n < P; ++n) {
                const double sc = which == 0 ? pow(h, n) : pow(h, -(n + 1));
                for (int m = 0; m <= n; ++m) {
                    const int t = n * (n + 1) / 2 + m;
                    double re = 0.0, im = 0.0;
                    if (ok) {
                        const float *src = v.data() + (size_t)g * PP;
                        re = src[m == 0 ? n * n : n * n + 2 * m - 1] * sc;
                        im = m == 0 ? 0.0 : src[n * n + 2 * m] * sc;
                    }
                    c[2 * t] = re;
                    c[2 * t + 1] = im;
                }
            }
        }
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "export copy");
}

int gbfmm_export_adaptive_tree(gbfmm_ctx *ctx, double *origin_side, int64_t *ncells, int32_t *level, uint64_t *key,
                               int32_t *begin, int32_t *count, int32_t *parent, uint32_t *perm)
{
    if (!ctx) return GBFMM_EINVAL;
    if (!ctx->have_last || !ctx->last_adaptive) return fail(ctx, GBFMM_EINVAL, "no adaptive evaluation to export");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    return export_adaptive_tree(ctx, origin_side, ncells, level, key, begin, count, parent, perm);
}

int gbfmm_selftest_wait(gbfmm_ctx *ctx, double limit_ms, void *stream)
{
    if (!ctx || !(limit_ms > 0.0) || limit_ms > 2000.0) return GBFMM_EINVAL;
    cudaSetDevice(ctx->device);
    launch_wait_selftest((uint64_t)(limit_ms * 1e6), ctx->d_status, static_cast<cudaStream_t>(stream));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "self-test launch");
}

int gbfmm_last_launch_count(const gbfmm_ctx *ctx, int64_t *count)
{
    if (!ctx || !count) return GBFMM_EINVAL;
    *count = ctx->launches_last;
    return GBFMM_OK;
}

int gbfmm_stage_times(gbfmm_ctx *ctx, float *ms, int max, int *count)
{
    if (!ctx || !ms) return GBFMM_EINVAL;
    if (!ctx->timed_last) return fail(ctx, GBFMM_EINVAL, "last evaluation was not timed");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->ev[9]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event sync");
    float t9[9];
    for (int k = 0; k < 9; ++k) {
        t9[k] = 0.f;
        cudaEventElapsedTime(&t9[k], ctx->ev[k], ctx->ev[k + 1]);
    }
    if (ctx->stage_order_last == 1) std::swap(t9[7], t9[8]);  // reported as 7 L2P, 8 P2P
    if (ctx->stage_order_last == 2) {
        float l2p = 0.f, p2p = 0.f;
        cudaEventElapsedTime(&l2p, ctx->ev_aux[2], ctx->ev[9]);
        cudaEventElapsedTime(&p2p, ctx->ev_aux[0], ctx->ev_aux[1]);
        t9[7] += l2p;  // ev 7 -> 8: what ran on the far stream before the join (adaptive: M2P)
        t9[8] = p2p;
    }
    int k = 0;
    for (; k < 9 && k < max; ++k) ms[k] = t9[k];
    if (k < max) {
        float t = 0.f;
        if (ctx->ops_built_last) cudaEventElapsedTime(&t, ctx->ev[kStages], ctx->ev[0]);
        ms[k++] = t;
    }
    if (count) *count = k;
    return GBFMM_OK;
}

}  // extern "C"
