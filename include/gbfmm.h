/*
 * gbfmm.h -- C ABI of the GB300-native Laplace FMM / treecode library (libgbfmm.so).
 *
 * The library evaluates, for N point charges (or masses) x_j with strengths q_j,
 *     phi_i      = sum_{j != i} q_j / |x_i - x_j|
 *     grad phi_i = -sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3
 * which is Eq. 1 of Yokota & Barba, "Treecode and fast multipole method for
 * N-body simulation with CUDA", without the target mass m_i: the quantity their
 * P2P kernel (Listing 1) accumulates.  Gravitational acceleration is +grad phi,
 * the electrostatic field is -grad phi; the caller chooses.
 *
 * The far field is approximated by the fast multipole method (Section "Fast
 * N-body simulation": P2M, M2M, M2L, L2L, L2P; Eq. 2-9) or by the treecode (P2M,
 * M2M, M2P over the same interaction lists), the near field by the direct P2P
 * sum over the 27 neighbouring leaf cells.
 *
 * Conventions shared by every call:
 *   - device pointers are CUDA global-memory addresses on the context's device;
 *     host pointers are ordinary host memory;
 *   - particle arrays are float32, 4 per particle: (x, y, z, q); outputs are
 *     float32, 4 per particle: (phi, dphi/dx, dphi/dy, dphi/dz), in the caller's
 *     original particle order;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     device work is enqueued on it and the call returns without waiting unless
 *     the call's description says otherwise;
 *   - every call returns a gbfmm_status; no exception crosses the ABI; after an
 *     error the context stays usable and gbfmm_last_error() describes it;
 *   - a context is not thread-safe: use it from one host thread and one stream
 *     at a time.
 */
#ifndef GBFMM_H
#define GBFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBFMM_VERSION 1

typedef enum gbfmm_status {
    GBFMM_OK = 0,
    GBFMM_EINVAL = 1,      /* null pointer, n < 0, non-finite coordinate, bad parameter */
    GBFMM_ENOMEM = 2,      /* workspace too small, or a library allocation failed */
    GBFMM_ECUDA = 3,       /* a CUDA runtime call failed (message in gbfmm_last_error) */
    GBFMM_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    GBFMM_EUNSUPPORTED = 5 /* order p or tree depth not compiled in */
} gbfmm_status;

enum { GBFMM_METHOD_FMM = 0, GBFMM_METHOD_TREECODE = 1 };
enum { GBFMM_TREE_UNIFORM = 0, GBFMM_TREE_ADAPTIVE = 1 };
/* list kinds: the uniform tree's P2P and M2L lists; the adaptive tree's U (P2P), V (M2L),
 * W (M2P) and X (P2L) lists */
enum {
    GBFMM_LIST_P2P = 0,
    GBFMM_LIST_M2L = 1,
    GBFMM_LIST_U = 2,
    GBFMM_LIST_V = 3,
    GBFMM_LIST_W = 4,
    GBFMM_LIST_X = 5
};

/* flags */
#define GBFMM_FLAG_STAGE_TIMING 1 /* record CUDA events between stages (gbfmm_stage_times) */
/* run M2L on the FP32 CUDA cores instead of the tcgen05 tensor cores (FP16 operands split in
 * three products with FP32 accumulation; the default).  Both compute Eq. 4 over the same
 * admissible pairs; they differ by rounding only. */
#define GBFMM_FLAG_M2L_CUDA_CORES 2
/* run every stage on the caller's stream, one after another.  By default an FMM evaluation
 * runs the near field (P2P, Listings 1-2) on a low-priority stream of the context while the
 * expansions (P2M .. L2L) run on a high-priority one, both forked from and joined back into the
 * caller's stream (event waits only, so stream capture sees one graph); the output is the same
 * bit for bit. */
#define GBFMM_FLAG_SERIAL 4
/* run the M2L as the list-based tensor-core kernel (128 target cells per CTA, sources gathered
 * through the M2L / V list) instead of the default block form (one GEMM per parent offset:
 * over all parents of a level on the uniform tree, over the cells with children on the adaptive
 * tree, whose colleagues' children are gathered).  Same Eq. 4, same precision scheme; they
 * differ by rounding only. */
#define GBFMM_FLAG_M2L_GATHERED 8
/* uniform tree: run the M2L by rotation to the translation axis on the FP32 CUDA cores: per
 * list entry, rotate the source expansion so that the offset lies on +z, translate along z
 * (equal orders only), rotate back -- O(p^3) per pair instead of the dense operator's O(p^4)
 * (the rotation-based M2L of the FMM literature; Section "Overview of Advanced Techniques").
 * The factors are computed on the host in FP64 and checked against the dense operators at the
 * first use of an order (synchronous, ECUDA if the check fails).  Ignored by the adaptive tree
 * and the treecode; GBFMM_FLAG_M2L_CUDA_CORES takes precedence. */
#define GBFMM_FLAG_M2L_ROTATION 16

/*
 * Parameters of one evaluation (Section "Fast N-body simulation").
 *   p          expansion order in the paper's convention: degrees n = 0..p-1
 *              (Eq. 4 sums n up to p-1); compiled orders: 4, 6, 8, 10.
 *   leaf_size  uniform tree: depth L = the smallest L >= 0 with
 *              n <= leaf_size * 8^L (mean leaf occupancy <= leaf_size); the paper
 *              keeps the number of cells proportional to N.  L <= 10.
 *              adaptive tree: a cell splits while it holds more than leaf_size
 *              particles, down to level 21 at most.
 *   tree       GBFMM_TREE_UNIFORM: every level of the octree is dense (Section
 *              "Fast N-body simulation"; the paper's own experiments);
 *              GBFMM_TREE_ADAPTIVE: the adaptive octree of the FMM of Cheng,
 *              Greengard & Rokhlin (1999), which the paper cites for its
 *              translation operators, with its U, V, W, X lists.
 *   method     GBFMM_METHOD_FMM or GBFMM_METHOD_TREECODE: the multipoles of the
 *              interaction list of a leaf and of its ancestors act on its
 *              particles by M2P; no local expansions.  On the adaptive tree the
 *              treecode takes M2P over W and over V of the leaf and its
 *              ancestors, and P2P over U and over X of the leaf and its
 *              ancestors (X cells are larger than the target and close to it).
 *   eps2       softening added to r^2 in P2P only (Listing 1's eps); pairs at
 *              exactly zero distance contribute nothing whatever eps2 is.
 *   has_box    0: root cube from the data (centre of the bounding box, side =
 *              its largest extent); 1: use box_origin / box_side (particles
 *              outside it are clamped into the boundary cells).
 *   flags      GBFMM_FLAG_* bits.
 */
typedef struct gbfmm_params {
    int32_t p;
    int32_t leaf_size;
    int32_t tree;
    int32_t method;
    double eps2;
    int32_t has_box;
    int32_t flags;
    double box_origin[3];
    double box_side;
} gbfmm_params;

typedef struct gbfmm_ctx gbfmm_ctx;

/* Library version (GBFMM_VERSION). */
int gbfmm_version(void);

/* Fill *prm with p = 10, leaf_size = 64, uniform tree, FMM, eps2 = 0, no box.
 * EINVAL if prm is NULL. */
int gbfmm_default_params(gbfmm_params *prm);

/* Create a context on CUDA device `device`.  The library allocates and owns the
 * context, a device status word and (lazily, per order p) the translation
 * operator tables (M2L: 343 x p^2 x p^2 floats, M2M and L2L: 8 x p^2 x p^2).
 * *out is NULL on failure.  ECUDA / ENOMEM on failure. */
int gbfmm_create(gbfmm_ctx **out, int device);

/* Free the context and everything it owns.  NULL-safe.  Waits for the device. */
int gbfmm_destroy(gbfmm_ctx *ctx);

/* Message describing the last error of this context ("" if none).  The string
 * is owned by the context and valid until the next call on it. */
const char *gbfmm_last_error(const gbfmm_ctx *ctx);

/* Plan an evaluation of n particles: tree depth and the device workspace size
 * gbfmm_evaluate needs (bytes, an upper bound independent of the particle
 * positions).  Either output pointer may be NULL.  For the adaptive tree the depth
 * is data dependent: *levels = 21 (the maximum) and *workspace_bytes = 0.
 * EINVAL / EUNSUPPORTED. */
int gbfmm_plan(const gbfmm_params *prm, int64_t n, int32_t *levels, size_t *workspace_bytes);

/*
 * Evaluate potential and gradient of n particles, fully on the device.
 *   d_xyzq       device, 4*n floats (x, y, z, q); read only.
 *   d_out        device, 4*n floats (phi, dphi/dx, dphi/dy, dphi/dz), written in
 *                the original order.  Must not alias d_xyzq.
 *   d_workspace  device scratch of at least gbfmm_plan's workspace_bytes, 256-byte
 *                aligned, owned by the caller; it holds the tree, lists and
 *                expansions of this evaluation until the next call that uses it.
 * Asynchronous on `stream`.  The first call with a new p also builds that order's
 * operator tables on the stream.  Non-finite coordinates are detected on the
 * device: the output is then undefined (but every access stays in bounds) and
 * gbfmm_sync_status reports EINVAL.  n = 0 returns OK without work.
 *
 * Adaptive tree: d_workspace and workspace_bytes are ignored (NULL / 0 allowed); the
 * tree, lists and expansions live in device buffers the context owns and grows on
 * demand.  The call sizes them from counts it reads back while it builds the tree,
 * so it synchronises `stream` several times and cannot be captured into a CUDA graph.
 */
int gbfmm_evaluate(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                   void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * Same evaluation from HOST buffers: copies h_xyzq to the device, evaluates,
 * copies the result to h_out and waits for the stream.  The device buffers and
 * workspace are allocated by the library, kept in the context and grown on
 * demand.  Returns the device status of the evaluation (as gbfmm_sync_status).
 */
int gbfmm_evaluate_host(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *h_xyzq, float *h_out,
                        void *stream);

/* Wait for `stream`, then return and clear the device status word: OK, EINVAL
 * (a non-finite coordinate was seen) or ETIMEOUT (a bounded wait gave up). */
int gbfmm_sync_status(gbfmm_ctx *ctx, void *stream);

/*
 * Direct O(N^2) evaluation on the device (Eq. 1 over all pairs; the paper's
 * "direct" curve of Fig. 4), same input/output layout and pair rules as
 * gbfmm_evaluate: d_src 4*n_src floats, d_tgt 4*n_tgt floats (q ignored),
 * d_out 4*n_tgt floats in target order.  No workspace.  Asynchronous.
 */
int gbfmm_direct(gbfmm_ctx *ctx, int64_t n_src, const float *d_src, int64_t n_tgt, const float *d_tgt, double eps2,
                 float *d_out, void *stream);

/*
 * Debug export of the last gbfmm_evaluate on this context (its workspace must
 * not have been reused).  All outputs are caller-owned HOST buffers; the calls
 * wait for the device.
 *
 * gbfmm_export_tree: origin_side[4] = root origin xyz and side (FP64);
 *   sorted_leaf_keys[n] = Morton key at depth L of each particle in sorted order
 *   (the 63-bit key shifted right by 3(21-L)); perm[n] = original index of the
 *   particle at each sorted position; begin[C], count[C] = particle range of every
 *   cell, C = (8^(L+1)-1)/7, cell of level l with key k at (8^l-1)/7 + k.
 *   Any pointer may be NULL to skip it.
 * gbfmm_export_lists: kind GBFMM_LIST_P2P (rows: the 8^L leaves) or
 *   GBFMM_LIST_M2L (rows: all C cells); offs[rows+1], ids[cap] = global cell
 *   indices, each row sorted ascending; *n_entries = entries.  ENOMEM if cap is
 *   too small (n_entries still set).
 * gbfmm_export_expansions: which = 0 multipole M, 1 local L; coef[C * p(p+1)]
 *   FP64 = for every cell the p(p+1)/2 complex coefficients (m >= 0, index
 *   n(n+1)/2+m, re/im interleaved) in the paper's unscaled normalisation (Eq. 2, 3).
 *   Levels the method does not form are zero.
 *   After an adaptive evaluation: gbfmm_export_tree returns EINVAL (use
 *   gbfmm_export_adaptive_tree); gbfmm_export_lists takes GBFMM_LIST_U, _V, _W or
 *   _X with rows = the adaptive tree's cells; gbfmm_export_expansions writes the
 *   adaptive tree's cells (levels 0 and 1 are zero).
 */
int gbfmm_export_tree(gbfmm_ctx *ctx, double *origin_side, uint32_t *sorted_leaf_keys, uint32_t *perm,
                      int32_t *begin, int32_t *count);
int gbfmm_export_lists(gbfmm_ctx *ctx, int kind, int32_t *offs, int32_t *ids, int64_t cap, int64_t *n_entries);
int gbfmm_export_expansions(gbfmm_ctx *ctx, int which, double *coef);

/*
 * Debug export of the last adaptive evaluation (GBFMM_TREE_ADAPTIVE).  Host buffers, any
 * may be NULL; call once with only ncells to size them.  Cells are numbered level by
 * level, in key order within a level (root = 0).  origin_side[4] as gbfmm_export_tree;
 * *ncells = number of cells C; level[C]; key[C] = the cell's Morton key at its level (the
 * 63-bit particle key shifted right by 3(21 - level)); begin[C], count[C] = its particle
 * range in sorted order; parent[C] (-1 for the root); perm[n] = original index of each
 * sorted position (particles sorted by their full 63-bit key, ties by original index).
 * EINVAL if the last evaluation was not adaptive.  Waits for the device.
 */
int gbfmm_export_adaptive_tree(gbfmm_ctx *ctx, double *origin_side, int64_t *ncells, int32_t *level, uint64_t *key,
                               int32_t *begin, int32_t *count, int32_t *parent, uint32_t *perm);

/*
 * Per-stage device times (ms) of the last evaluate run with
 * GBFMM_FLAG_STAGE_TIMING, in this order: 0 box+keys, 1 sort, 2 cells+lists,
 * 3 P2M, 4 M2M, 5 M2L (or M2P), 6 L2L, 7 L2P(+output), 8 P2P, 9 operator build
 * (0 when cached).  When P2P ran on the context's second stream (the default for the FMM),
 * stage 8 is its own duration, overlapping stages 3-6, and the stages add up to more than the
 * evaluation took; with GBFMM_FLAG_SERIAL they are consecutive.  Waits for the device.
 * *count = stages written (<= max).
 */
int gbfmm_stage_times(gbfmm_ctx *ctx, float *ms, int max, int *count);

/* Test of the bounded device waits (no counterpart in the paper): enqueues one CTA that waits
 * on an mbarrier no thread arrives on, with the same bounded-wait routine the M2L and P2P pipelines
 * use, limited to limit_ms (0 < limit_ms <= 2000).  When it gives up it raises the context's
 * status word, so the next gbfmm_sync_status returns ETIMEOUT; the context stays usable.
 * Asynchronous on `stream`.  EINVAL / ECUDA. */
int gbfmm_selftest_wait(gbfmm_ctx *ctx, double limit_ms, void *stream);

/* Number of library kernels the last gbfmm_evaluate / gbfmm_evaluate_host / gbfmm_direct
 * on this context enqueued (operator-table builds included; runtime memsets excluded). */
int gbfmm_last_launch_count(const gbfmm_ctx *ctx, int64_t *count);

/*
 * Allocation-free Morton sort (no counterpart in the paper: it exists for callers that may
 * not allocate device memory -- code whose host framework owns every device byte, plug-ins
 * handed only their input and output buffers, hooks that run where allocation is forbidden).
 * It runs the tree front end of gbfmm_evaluate -- root box, depth-L Morton keys (L from
 * prm->leaf_size as in gbfmm_plan; prm is validated like gbfmm_plan), the stable radix sort
 * by (leaf key, original index) and the gather -- with no context and no cudaMalloc, cudaFree
 * or allocating library call.
 *   d_xyzq              device, 4*n floats, 16-byte aligned, read only
 *   d_sorted_xyzq       device, 4*n floats, 16-byte aligned: particles in sorted order
 *   d_perm              device, n uint32: original index of each sorted position
 *   d_sorted_leaf_keys  device, n uint32: depth-L Morton key of each sorted position
 *   d_status            device, one int32, or NULL: cleared by the call, then raised by its
 *                       kernels -- bit 0 (value 1) a non-finite coordinate was seen (it is
 *                       clamped into a boundary cell), bit 1 (value 2) a bounded device wait
 *                       gave up (the outputs are then invalid).  Read it after the stream
 *                       completes.  With NULL these conditions are not reported.
 * The outputs equal what gbfmm_export_tree reports after gbfmm_evaluate with the same prm.
 * No two of the five buffers may share a byte (EINVAL otherwise).
 * Uniform tree only (prm->tree == GBFMM_TREE_UNIFORM; EUNSUPPORTED otherwise, before any
 * launch): its keys have 3L <= 30 bits.
 * Scratch: one static device array (about 8.4 MB) per GPU that loads the library, held
 * until the process exits; n is limited to 1,048,576 (EUNSUPPORTED beyond).  The first call
 * on a device looks the array's address up (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture.  The address is cached for the life of the
 * process: calls after cudaDeviceReset on that device are not supported.  Every call clears
 * the scratch words that must start at zero; calls that overlap on the GPU share the array
 * and race.  n = 0 returns OK without work (d_status untouched).  Asynchronous on `stream`;
 * EINVAL / EUNSUPPORTED / ECUDA.
 */
int gbfmm_sort_static(const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_sorted_xyzq, uint32_t *d_perm,
                      uint32_t *d_sorted_leaf_keys, int32_t *d_status, void *stream);

/*
 * Multi-instance engine: batched evaluation of many independent particle sets and a served
 * request stream with continuous batching (the paper evaluates one system at a time; this is
 * the runtime around the same single-instance evaluation).
 *
 * The engine owns `workers` host threads; each has its own context (operator tables, adaptive
 * tree buffers), CUDA stream, device input/output buffers and uniform-tree workspace, kept
 * resident and grown on demand.  Requests wait in one FIFO queue; a free worker takes the
 * head request when the footprints of the running requests plus its own fit in
 * memory_budget_bytes (a request larger than the whole budget runs alone).  Requests on
 * different workers overlap on the device; each runs gbfmm_evaluate unchanged, so its result
 * is the same alone or in a mix.  Footprint estimate: uniform tree 32 B x n (inputs and
 * outputs, served requests only) + gbfmm_plan's workspace; adaptive tree 32 B x n + 128 B x n +
 * (4n / leaf_size + 64) x (8p^2 + 640) B.  The workers' resident buffers are not released
 * between requests, so the budget bounds what running requests use, not the engine's peak.
 *
 * gbfmm_engine_create: 1 <= workers <= 64.  ECUDA / ENOMEM / EINVAL.
 * gbfmm_engine_destroy: stops the workers after their current request; requests still queued
 *   are dropped (their tickets become invalid).  NULL-safe.
 * gbfmm_engine_prepare: builds the operator tables of the listed orders on every worker (one
 *   small evaluation each), so that no later request pays for them.  Synchronous.
 * gbfmm_engine_submit: queues one request; h_xyzq (4n floats) and h_out (4n floats) are HOST
 *   buffers that must stay valid until gbfmm_engine_wait returns for the ticket.  Returns at
 *   once with *ticket.  prm is copied (GBFMM_FLAG_STAGE_TIMING is ignored).
 * gbfmm_engine_wait: waits up to timeout_ms for the ticket; on completion returns OK and sets
 *   *status (the request's gbfmm status), *queue_ms (submit -> start) and *latency_ms
 *   (submit -> result in h_out), then forgets the ticket.  ETIMEOUT if it is not done yet
 *   (the ticket stays valid); EINVAL for an unknown ticket.  Any output pointer may be NULL.
 * gbfmm_engine_run_batch: evaluates nb instances whose particles are DEVICE arrays: instance
 *   i is d_xyzq + 4*offsets[i] .. 4*offsets[i+1] (floats; offsets is a host array of nb + 1
 *   ascending entries), results at the same offsets of d_out; prm[i] its parameters (host
 *   array).  Returns when all are done; status[i] (host, may be NULL) receives each one's
 *   status; the return value is the first error.  Must not be mixed with served requests whose
 *   tickets another thread is waiting on.
 */
typedef struct gbfmm_engine gbfmm_engine;
int gbfmm_engine_create(gbfmm_engine **out, int device, int32_t workers, size_t memory_budget_bytes);
int gbfmm_engine_destroy(gbfmm_engine *e);
int gbfmm_engine_prepare(gbfmm_engine *e, const int32_t *orders, int32_t norders);
int gbfmm_engine_submit(gbfmm_engine *e, const gbfmm_params *prm, int64_t n, const float *h_xyzq, float *h_out,
                        int64_t *ticket);
int gbfmm_engine_wait(gbfmm_engine *e, int64_t ticket, double timeout_ms, int32_t *status, double *queue_ms,
                      double *latency_ms);
int gbfmm_engine_run_batch(gbfmm_engine *e, int32_t nb, const int64_t *offsets, const gbfmm_params *prm,
                           const float *d_xyzq, float *d_out, int32_t *status);

/*
 * Repeated evaluations and tuning (no counterpart in the paper; for time-stepping codes and
 * for the batched and served forms).
 *
 * gbfmm_graph_create: captures one uniform-tree gbfmm_evaluate (same arguments) into a CUDA
 *   graph and instantiates it; an eager evaluation runs first (it builds the order's operator
 *   tables and checks the arguments) and must succeed.  The graph replays the evaluation of the
 *   same buffers: the caller may change the contents of d_xyzq (n, the pointers and prm stay)
 *   between launches.  It uses the context's operator tables, status word and scratch: destroy
 *   it before the context, and read errors with gbfmm_sync_status as after gbfmm_evaluate.
 *   EUNSUPPORTED for the adaptive tree (its evaluation reads counts back from the device).
 * gbfmm_graph_launch: one replay, asynchronous on `stream`.
 * gbfmm_graph_destroy: NULL-safe.
 * gbfmm_tune_leaf: leaf-size autotuner.  For each of the ncand leaf sizes in candidates (host
 *   array) it times one evaluation of the caller's particles d_xyzq (device, 4n floats; read
 *   only) after one warm-up, with prm's other fields, into the context's own device buffers;
 *   *best_leaf receives the fastest candidate and *best_ms (may be NULL) its time.
 *   Synchronous.  Candidates that gbfmm_plan rejects are skipped; EINVAL if none is valid.
 * gbfmm_tune: the same over every pair of a leaf size (leaf_candidates) and a P2P launch shape
 *   (lpc_candidates: target leaves per CTA of the P2P kernel, 0 .. 64, 0 = the library's
 *   choice; n_lpc = 0 keeps the context's setting).  *best_leaf and *best_lpc (may be NULL)
 *   receive the fastest pair and *best_ms its time; the context keeps best_lpc for its later
 *   evaluations (as gbfmm_set_p2p_leaves_per_cta).  The leaf size is the caller's to apply.
 * gbfmm_set_p2p_leaves_per_cta: this context's P2P launch shape, 0 .. 64 target leaves per CTA
 *   (0 = the library's choice, 4).  Every leaf's sums are formed the same way whichever CTA
 *   takes it, so results are bit-identical for every setting; only the time changes.  EINVAL.
 */
typedef struct gbfmm_graph gbfmm_graph;
int gbfmm_graph_create(gbfmm_graph **out, gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq,
                       float *d_out, void *d_workspace, size_t workspace_bytes);
int gbfmm_graph_launch(gbfmm_graph *g, void *stream);
int gbfmm_graph_destroy(gbfmm_graph *g);
int gbfmm_tune_leaf(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, const int32_t *candidates,
                    int32_t ncand, int32_t *best_leaf, float *best_ms);
int gbfmm_tune(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, const int32_t *leaf_candidates,
               int32_t n_leaf, const int32_t *lpc_candidates, int32_t n_lpc, int32_t *best_leaf, int32_t *best_lpc,
               float *best_ms);
int gbfmm_set_p2p_leaves_per_cta(gbfmm_ctx *ctx, int32_t leaves);

/*
 * Batched evaluation: nb independent instances (uneven N, orders, trees) in one CUDA graph.
 * Instance i is d_xyzq + 4*offsets[i] .. 4*offsets[i+1] (floats, DEVICE; offsets is a HOST array
 * of nb + 1 ascending entries from >= 0), its result at the same offsets of d_out (which must not
 * overlap d_xyzq), prm[i] (host array) its parameters; GBFMM_FLAG_SERIAL is forced and
 * GBFMM_FLAG_STAGE_TIMING ignored.  The instances share no state but the context's operator
 * tables and status word.
 *
 * gbfmm_batch_create: evaluates every instance once with counts read back (synchronous; the
 *   outputs are then valid), lays each adaptive instance out for capacities above its tree's
 *   and lists' counts (twice the cells and leaves, levels down to three below the deepest, lists
 *   in proportion to the cells with half again as margin, V rows up to 189 per cell),
 *   evaluates it once more that way, and captures
 *   all of them into one graph whose `lanes` concurrent branches (1..64) take the instances by
 *   particle count, largest first, each lane running its instances one after another.  In the
 *   graph every adaptive stage reads its counts on the device: no host synchronisation, no
 *   allocation.  The batch owns the instances' trees, lists, expansions and uniform workspaces
 *   (device memory of the order of the sum of the instances' own).  Adaptive leaf sizes above
 *   16384 are EUNSUPPORTED.  EINVAL / ENOMEM / ECUDA / EUNSUPPORTED.
 * gbfmm_batch_launch: one replay on `stream`, asynchronous: it evaluates the particles the
 *   arrays hold at that time (same pointers, counts and parameters).  An adaptive instance whose
 *   tree or lists outgrow its capacities (the caller moved its particles far) leaves its output
 *   unwritten and the next gbfmm_sync_status returns ENOMEM: re-create the batch.
 * gbfmm_batch_info: *lanes and the number of kernel nodes of the graph (either may be NULL).
 * gbfmm_batch_destroy: waits for the device and frees the batch.  NULL-safe.  Destroy it before
 *   its context.
 * gbfmm_evaluate_batch: the same through a batch the context keeps: the first call with a given
 *   (nb, offsets, prm, d_xyzq, d_out) creates it with 64 lanes (that call is synchronous),
 *   later calls with the same arguments only launch its graph on `stream`.
 */
typedef struct gbfmm_batch gbfmm_batch;
int gbfmm_batch_create(gbfmm_batch **out, gbfmm_ctx *ctx, int32_t nb, const int64_t *offsets, const gbfmm_params *prm,
                       const float *d_xyzq, float *d_out, int32_t lanes);
int gbfmm_batch_launch(gbfmm_batch *b, void *stream);
int gbfmm_batch_info(const gbfmm_batch *b, int32_t *lanes, int64_t *kernel_nodes);
int gbfmm_batch_destroy(gbfmm_batch *b);
int gbfmm_evaluate_batch(gbfmm_ctx *ctx, int32_t nb, const int64_t *offsets, const gbfmm_params *prm,
                         const float *d_xyzq, float *d_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBFMM_H */
