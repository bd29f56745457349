// Internal: the library context shared by the host-side translation units (api.cu for the
// uniform tree, adaptive.cu for the adaptive tree).  Not part of the C ABI.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"
#include "gbfmm.h"

namespace gbfmm {

constexpr int kBoxPartials = 304 * 8;
constexpr int kStages = 10;
constexpr int kOrders[4] = {4, 6, 8, 10};
constexpr int kAdaptiveMaxLevel = 21;  // 63-bit keys: 21 bits per axis

struct OpsCache {
    int P = 0;
    float *m2l = nullptr, *m2m = nullptr, *l2l = nullptr;
    void *m2l_f16 = nullptr;  // FP16 tensor-core operator blocks (hi | lo) + per-code scales (list-based M2L)
    void *m2l_blk = nullptr;
    void *m2l_rot = nullptr;  // rotation factors of the M2L operators (GBFMM_FLAG_M2L_ROTATION)  // uniform tree: per parent offset, the 8p^2 x 8p^2 FP16 blocks (hi | lo) + scale
    bool built = false;
};

// a device buffer owned by the context, grown on demand
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    template <class T>
    T *as() const
    {
        return static_cast<T *>(p);
    }
};

// Sizes of an adaptive evaluation: the counts an evaluation read back (exact), or the
// capacities a captured evaluation is laid out for.  level[l]: cells of level l; list: U, V,
// W, X entries; chain: the treecode's two chain-list totals; maxl: deepest level.
struct AdaptCaps {
    int64_t cells = 0, leaves = 0;
    int64_t level[kAdaptiveMaxLevel + 1] = {};
    int64_t list[4] = {}, chain[2] = {};
    int32_t maxl = 0;
    bool valid = false;
};

// device state of the last adaptive evaluation (all buffers owned by the context)
struct AdaptiveState {
    DevBuf keys0, keys1, idx0, idx1, sx, far, hist, scan_tmp, flags, scan, pcell, leaf_of, box;
    DevBuf level, key, begin, count, end, parent, child_begin, nchild, child_of, coll;
    DevBuf lcnt[4], loffs[4], lids[4], vcode;  // U, V, W, X
    DevBuf M, Lc, tlist, tdesc, leaves, group_cnt, cscale, geom;  // geom: float4 (centre, 1/h) per cell
    DevBuf info;                                                   // small device-side totals read by the host
    DevBuf anchor;                                                 // int4 integer box per cell (depth 21)
    DevBuf presplit;                                               // FP16 pre-split source rows (gathered M2L)
    DevBuf near;                                                   // P2P's compensated sums, 2 float4 per particle
    DevBuf tc_cnt, tc_offs[2], tc_ids[2];  // treecode rows: [0] U + ancestors' X, [1] W + ancestors' V
    // block-form M2L: unit flags and their scan, unit of every cell, the units, their count, the
    // pre-split rows and scales, the colleague rows per (tile, offset), the offset ranges' partial sums
    DevBuf ab_flag, ab_scan, ab_unit_of, ab_units, ab_nu, ab_pre, ab_scale, ab_src, lpart;
    DevBuf partials;  // root-box reduction scratch of evaluations that do not use the context's
    AdaptCaps counts;  // the sizes the last host-counted evaluation read back
    int64_t n = 0, ncells = 0, nleaves = 0, entries[4] = {0, 0, 0, 0};
    int P = 0, max_level = 0;
    std::vector<int> level_start;
    uint64_t *skeys = nullptr;
    uint32_t *perm = nullptr;
};

}  // namespace gbfmm

struct gbfmm_ctx {
    int device = 0;
    int p2p_leaves_per_cta = 0;  // P2P launch shape (0: the library's choice)
    std::string err;
    int *d_status = nullptr;
    unsigned *d_counter = nullptr;
    float *d_partials = nullptr;
    float *d_zero = nullptr;
    gbfmm::OpsCache ops[4];
    // last evaluation
    bool have_last = false;
    bool last_adaptive = false;
    gbfmm::Layout last{};
    unsigned char *last_ws = nullptr;
    size_t last_keys = 0, last_idx = 0;
    int last_method = 0;
    bool last_m2l_lists = true;  // the last uniform evaluation built its M2L rows
    gbfmm::AdaptiveState ad;
    // host-buffer path
    float *h_in = nullptr, *h_out = nullptr;
    void *h_ws = nullptr;
    int64_t h_cap_n = 0;
    size_t h_ws_bytes = 0;
    // stage timing
    cudaEvent_t ev[gbfmm::kStages + 1] = {};
    bool timed_last = false;
    // order of the last timed evaluation's stages 7 (L2P) and 8 (P2P): 0 = L2P then P2P (ev 7, 8,
    // 9); 1 = P2P then L2P, serial; 2 = P2P on s_near between ev_aux[0] and ev_aux[1] while the
    // far field ran on s_far, whose L2P (after the join on ev_aux[2]) ends at ev[9]
    int stage_order_last = 0;
    // the near field runs beside the far field: P2P on s_near (lowest priority), M2L .. L2P on
    // s_far (highest), forked from and joined into the caller's stream by events
    cudaStream_t s_far = nullptr, s_near = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_near = nullptr, ev_join = nullptr;
    cudaEvent_t ev_aux[3] = {};
    bool ops_built_last = false;
    int64_t launches_last = 0;
    // gbfmm_evaluate_batch: the captured batch of the last call and the arguments it was made for
    gbfmm_batch *batch = nullptr;
    std::vector<int64_t> batch_offsets;
    std::vector<gbfmm_params> batch_prm;
    const float *batch_x = nullptr;
    float *batch_out = nullptr;
};

namespace gbfmm {
int order_slot(int p);
int fail(gbfmm_ctx *ctx, int code, const std::string &msg);
int cuda_fail(gbfmm_ctx *ctx, cudaError_t e, const char *what);
int ensure_ops(gbfmm_ctx *ctx, int P, cudaStream_t s, bool *built_now);
// the block operators of the M2L's block form (both trees), built on the stream at first use
int ensure_blk(gbfmm_ctx *ctx, int P, cudaStream_t s);
int64_t launch_count();
// adaptive tree (adaptive.cu)
int evaluate_adaptive(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                      cudaStream_t s);
// The same evaluation into the state A.  caps == nullptr: sized from counts read back (A.counts
// receives them).  caps given: no host read, no synchronisation and (after a first call with the
// same caps) no allocation, so the call can be captured into a CUDA graph; every launch covers
// the capacities and reads the counts on the device, and a tree or list that outgrows them
// raises kStatusCapacity and skips the rest of the evaluation.  partials / counter: the root-box
// reduction scratch (kBoxPartials floats, one zeroed unsigned) of this evaluation.
int evaluate_adaptive_in(gbfmm_ctx *ctx, AdaptiveState &A, const AdaptCaps *caps, const gbfmm_params *prm,
                         int64_t n, const float *d_xyzq, float *d_out, cudaStream_t s, float *partials,
                         unsigned *counter);
// the uniform-tree evaluation (api.cu) with its root-box reduction scratch given
int evaluate_uniform_in(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                        void *d_workspace, size_t workspace_bytes, cudaStream_t s, float *partials,
                        unsigned *counter);
int export_adaptive_tree(gbfmm_ctx *ctx, double *origin_side, int64_t *ncells, int32_t *level, uint64_t *key,
                         int32_t *begin, int32_t *count, int32_t *parent, uint32_t *perm);
int export_adaptive_expansions(gbfmm_ctx *ctx, int which, double *coef);
int export_adaptive_list(gbfmm_ctx *ctx, int kind, int32_t *offs, int32_t *ids, int64_t cap, int64_t *n_entries);
void free_adaptive(AdaptiveState &a);
}  // namespace gbfmm
