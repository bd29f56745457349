// Adaptive octree FMM on the device (the adaptive FMM of Cheng, Greengard & Rokhlin 1999,
// which the paper cites for its translation operators).
//
// Tree: the particles are sorted by their full 63-bit Morton key (stable radix sort), then
// the tree is built level by level: a cell splits while it holds more than leaf_size particles
// (and is above level 21); only nonempty children exist.  Cells are numbered level by level,
// in key order within a level.  Every level is one flag / scan / compact round over the
// particles; the host reads the number of new cells after each round to size the cell arrays.
//
// Lists (every cell B):
//   colleagues(B)  cells of B's level adjacent to B (B included), stored by position (27 slots)
//   U(B), leaf     leaves adjacent to B, any level (P2P)
//   V(B)           children of the colleagues of B's parent not adjacent to B (M2L), in
//                  ascending stencil code, the code stored beside the id
//   W(B), leaf     descendants of B's colleagues whose parent is adjacent to B but which are not
//                  (M2P; the descent stops there)
//   X(B)           leaves C with B in W(C): leaf colleagues of B's strict ancestors that are
//                  adjacent to B's parent but not to B (P2L)
// Adjacency is exact on integer boxes at depth 21 (boxes that touch or overlap).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "context.h"

namespace gbfmm {

constexpr int kAdaptMaxLevel = kAdaptiveMaxLevel;
constexpr int kListU = 0, kListV = 1, kListW = 2, kListX = 3;
constexpr int kDescentStack = 256;

// ---- keys ---------------------------------------------------------------------------------
__global__ void k_keys64(const float4 *__restrict__ x, int64_t n, const Box *__restrict__ box,
                         uint64_t *__restrict__ keys, uint32_t *__restrict__ idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Box b = *box;
    float4 p = __ldg(&x[i]);
    float c[3] = {p.x, p.y, p.z};
    uint64_t k[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double t = __dsub_rn((double)c[d], b.origin[d]);
        double v = __dmul_rn(t, b.key_scale);
        double f = floor(v);
        if (!(f >= 0.0)) f = 0.0;
        if (f > 2097151.0) f = 2097151.0;
        k[d] = (uint64_t)f;
    }
    keys[i] = morton63(k[0], k[1], k[2]);
    idx[i] = (uint32_t)i;
}

// ---- tree construction --------------------------------------------------------------------
__global__ void k_tree_root(int64_t n, int32_t *level, uint64_t *key, int32_t *begin, int32_t *count,
                            int32_t *parent, int32_t *child_begin, int32_t *nchild, int32_t *child_of)
{
    level[0] = 0;
    key[0] = 0;
    begin[0] = 0;
    count[0] = (int32_t)n;
    parent[0] = -1;
    child_begin[0] = 0x7fffffff;
    nchild[0] = 0;
    for (int c = 0; c < 8; ++c) child_of[c] = -1;
}

__global__ void k_tree_pcell_init(int64_t n, int32_t *pcell)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) pcell[i] = 0;
}

// level l -> l + 1: a particle starts a new child when its cell splits and its level-(l+1)
// prefix differs from its predecessor's; particles of cells that do not split are done
__global__ void k_tree_flags(int64_t n, const uint64_t *__restrict__ sk, int l, int leaf_size, int max_level,
                             int32_t *__restrict__ pcell, const int32_t *__restrict__ count,
                             const int32_t *__restrict__ begin, uint32_t *__restrict__ flags,
                             int32_t *__restrict__ leaf_of)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t c = pcell[i];
    uint32_t f = 0;
    if (c >= 0) {
        if (count[c] > leaf_size && l < max_level) {
            const int sh = 3 * (kAdaptMaxLevel - (l + 1));
            f = (i == begin[c] || (sk[i] >> sh) != (sk[i - 1] >> sh)) ? 1u : 0u;
        } else {
            leaf_of[i] = c;
            pcell[i] = -1;
        }
    }
    flags[i] = f;
}

__global__ void k_tree_new_cells(int64_t n, const uint64_t *__restrict__ sk, int l, const int32_t *__restrict__ pcell,
                                 const uint32_t *__restrict__ flags, const uint32_t *__restrict__ scan, int64_t base,
                                 int32_t *level, uint64_t *key, int32_t *begin, int32_t *parent, int32_t *child_begin,
                                 int32_t *nchild, int32_t *child_of)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    const int64_t id = base + scan[i];
    const int32_t c = pcell[i];
    const int sh = 3 * (kAdaptMaxLevel - (l + 1));
    const uint64_t k = sk[i] >> sh;
    level[id] = l + 1;
    key[id] = k;
    begin[id] = (int32_t)i;
    parent[id] = c;
    child_begin[id] = 0x7fffffff;
    nchild[id] = 0;
    for (int q = 0; q < 8; ++q) child_of[id * 8 + q] = -1;
    child_of[(int64_t)c * 8 + (int)(k & 7)] = (int32_t)id;
    atomicAdd(&nchild[c], 1);
    atomicMin(&child_begin[c] , (int32_t)id);
}

__global__ void k_tree_counts(int64_t base, int64_t nnew, const int32_t *__restrict__ begin,
                              const int32_t *__restrict__ parent, int32_t *__restrict__ count)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnew) return;
    const int64_t id = base + t;
    const int32_t p = parent[id];
    const int32_t end = (t + 1 < nnew && parent[id + 1] == p) ? begin[id + 1] : begin[p] + count[p];
    count[id] = end - begin[id];
}

__global__ void k_tree_pcell(int64_t n, const uint32_t *__restrict__ flags, const uint32_t *__restrict__ scan,
                             int64_t base, int32_t *__restrict__ pcell)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || pcell[i] < 0) return;
    pcell[i] = (int32_t)(base + scan[i] + flags[i] - 1);
}

__global__ void k_cell_end(int64_t nc, const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                           int32_t *__restrict__ end)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < nc) end[c] = begin[c] + count[c];
}

// ---- colleagues (positional: slot (dx+1) + 3(dy+1) + 9(dz+1)) -----------------------------
GB_DEV int slot27(int dx, int dy, int dz) { return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1); }

__global__ void k_colleagues(int64_t lo, int64_t hi, int l, const uint64_t *__restrict__ key,
                             const int32_t *__restrict__ parent, const int32_t *__restrict__ child_of,
                             int32_t *__restrict__ coll)
{
    int64_t b = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= hi) return;
    int32_t *out = coll + b * 27;
    if (l == 0) {
        for (int s = 0; s < 27; ++s) out[s] = -1;
        out[13] = (int32_t)b;
        return;
    }
    int x, y, z;
    demorton63(key[b], x, y, z);
    const int side = 1 << l;
    const int32_t *pc = coll + (int64_t)parent[b] * 27;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int nx = x + dx, ny = y + dy, nz = z + dz;
                int32_t r = -1;
                if (nx >= 0 && ny >= 0 && nz >= 0 && nx < side && ny < side && nz < side) {
                    const int32_t a = pc[slot27((nx >> 1) - (x >> 1), (ny >> 1) - (y >> 1), (nz >> 1) - (z >> 1))];
                    if (a >= 0) r = child_of[(int64_t)a * 8 + ((nx & 1) | ((ny & 1) << 1) | ((nz & 1) << 2))];
                }
                out[slot27(dx, dy, dz)] = r;
            }
}

// ---- lists --------------------------------------------------------------------------------
struct TreeView {
    const int32_t *level, *parent, *nchild, *child_of, *coll;
    const uint64_t *key;
};

GB_DEV void cell_box(const TreeView &t, int32_t c, int64_t lo[3], int64_t &size)
{
    int x, y, z;
    const int l = t.level[c];
    demorton63(t.key[c], x, y, z);
    size = int64_t(1) << (kAdaptMaxLevel - l);
    lo[0] = x * size;
    lo[1] = y * size;
    lo[2] = z * size;
}

GB_DEV bool adjacent(const TreeView &t, int32_t a, int32_t b)
{
    int64_t la[3], lb[3], sa, sb;
    cell_box(t, a, la, sa);
    cell_box(t, b, lb, sb);
    for (int d = 0; d < 3; ++d)
        if (la[d] > lb[d] + sb || lb[d] > la[d] + sa) return false;
    return true;
}

// Calls f(id, code) for every entry of list `kind` of cell b; returns false if a descent
// exceeded its stack (the row is then incomplete and the caller raises the status word).
template <class F>
GB_DEV bool for_each_entry(const TreeView &t, int kind, int32_t b, F f)
{
    const int l = t.level[b];
    if (kind == kListV) {
        if (l < 2) return true;
        int x, y, z;
        demorton63(t.key[b], x, y, z);
        const int side = 1 << l, cx = x & 1, cy = y & 1, cz = z & 1;
        const int32_t *pc = t.coll + (int64_t)t.parent[b] * 27;
        for (int oz = -2 - cz; oz <= 3 - cz; ++oz)
            for (int oy = -2 - cy; oy <= 3 - cy; ++oy)
                for (int ox = -2 - cx; ox <= 3 - cx; ++ox) {
                    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                    const int nx = x + ox, ny = y + oy, nz = z + oz;
                    if (nx < 0 || ny < 0 || nz < 0 || nx >= side || ny >= side || nz >= side) continue;
                    const int32_t a = pc[slot27((nx >> 1) - (x >> 1), (ny >> 1) - (y >> 1), (nz >> 1) - (z >> 1))];
                    if (a < 0) continue;
                    const int32_t s = t.child_of[(int64_t)a * 8 + ((nx & 1) | ((ny & 1) << 1) | ((nz & 1) << 2))];
                    if (s >= 0) f(s, m2l_code(ox, oy, oz));
                }
        return true;
    }
    if (kind == kListX) {
        const int32_t pb = t.parent[b];
        if (pb < 0) return true;
        for (int32_t anc = pb; anc >= 0; anc = t.parent[anc]) {
            const int32_t *ac = t.coll + (int64_t)anc * 27;
            for (int s = 0; s < 27; ++s) {
                const int32_t c = ac[s];
                if (c < 0 || c == anc || t.nchild[c] != 0) continue;
                if (adjacent(t, pb, c) && !adjacent(t, b, c)) f(c, 0);
            }
        }
        return true;
    }
    // U and W: leaves only
    if (t.nchild[b] != 0) return true;
    bool ok = true;
    const int32_t *bc = t.coll + (int64_t)b * 27;
    for (int s = 0; s < 27; ++s) {
        const int32_t a = bc[s];
        if (a < 0) continue;
        if (t.nchild[a] == 0) {
            if (kind == kListU) f(a, 0);
            continue;
        }
        int32_t stack[kDescentStack];
        int sp = 0;
        for (int q = 0; q < 8; ++q) {
            const int32_t c = t.child_of[(int64_t)a * 8 + q];
            if (c >= 0) stack[sp++] = c;
        }
        while (sp > 0) {
            const int32_t d = stack[--sp];
            if (adjacent(t, b, d)) {
                if (t.nchild[d] == 0) {
                    if (kind == kListU) f(d, 0);
                } else {
                    for (int q = 0; q < 8; ++q) {
                        const int32_t c = t.child_of[(int64_t)d * 8 + q];
                        if (c < 0) continue;
                        if (sp < kDescentStack)
                            stack[sp++] = c;
                        else
                            ok = false;
                    }
                }
            } else if (kind == kListW) {
                f(d, 0);
            }
        }
    }
    if (kind == kListU)
        for (int32_t anc = t.parent[b]; anc >= 0; anc = t.parent[anc]) {
            const int32_t *ac = t.coll + (int64_t)anc * 27;
            for (int s = 0; s < 27; ++s) {
                const int32_t c = ac[s];
                if (c < 0 || c == anc || t.nchild[c] != 0) continue;
                if (adjacent(t, b, c)) f(c, 0);
            }
        }
    return ok;
}

__global__ void k_alist_count(int kind, int64_t nc, TreeView t, uint32_t *__restrict__ cnt, int *status)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nc) return;
    uint32_t k = 0;
    if (!for_each_entry(t, kind, (int32_t)b, [&](int32_t, int) { ++k; })) atomicOr(status, kStatusTimeout);
    cnt[b] = k;
}

__global__ void k_alist_fill(int kind, int64_t nc, TreeView t, const uint32_t *__restrict__ offs,
                             int32_t *__restrict__ ids, uint16_t *__restrict__ codes)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nc) return;
    uint32_t e = offs[b];
    for_each_entry(t, kind, (int32_t)b, [&](int32_t s, int code) {
        ids[e] = s;
        if (codes) codes[e] = (uint16_t)code;
        ++e;
    });
}

// ---- M2L targets grouped by (level, child position) ----------------------------------------
__global__ void k_group_count(int64_t lo, int64_t nc, const int32_t *__restrict__ level,
                              const uint64_t *__restrict__ key, uint32_t *__restrict__ gcnt)
{
    int64_t c = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    atomicAdd(&gcnt[level[c] * 8 + (int)(key[c] & 7)], 1u);
}

__global__ void k_group_fill(int64_t lo, int64_t nc, const int32_t *__restrict__ level,
                             const uint64_t *__restrict__ key, uint32_t *__restrict__ gcur,
                             int32_t *__restrict__ tlist)
{
    int64_t c = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const uint32_t pos = atomicAdd(&gcur[level[c] * 8 + (int)(key[c] & 7)], 1u);
    tlist[pos] = (int32_t)c;
}

__global__ void k_leaf_list(int64_t nc, const int32_t *__restrict__ nchild, uint32_t *__restrict__ cursor,
                            int32_t *__restrict__ leaves)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc || nchild[c] != 0) return;
    leaves[atomicAdd(cursor, 1u)] = (int32_t)c;
}

// ---- host orchestration ---------------------------------------------------------------------
namespace {

unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int grow(DevBuf &b, size_t bytes, bool keep, size_t used, cudaStream_t s)
{
    if (b.cap >= bytes) return 0;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) return -1;
    if (keep && b.p && used) cudaMemcpyAsync(p, b.p, std::min(used, b.cap), cudaMemcpyDeviceToDevice, s);
    if (b.p) {
        cudaStreamSynchronize(s);
        cudaFree(b.p);
    }
    b.p = p;
    b.cap = want;
    return 0;
}

template <class T>
T read1(const void *dptr, cudaStream_t s)
{
    T v{};
    cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return v;
}

}  // namespace

void free_adaptive(AdaptiveState &a)
{
    DevBuf *all[] = {&a.keys0, &a.keys1, &a.idx0, &a.idx1, &a.sx, &a.far, &a.hist, &a.scan_tmp, &a.flags, &a.scan,
                     &a.pcell, &a.leaf_of, &a.box, &a.level, &a.key, &a.begin, &a.count, &a.end, &a.parent,
                     &a.child_begin, &a.nchild, &a.child_of, &a.coll, &a.vcode, &a.M, &a.Lc, &a.tlist, &a.tdesc,
                     &a.leaves, &a.group_cnt, &a.cscale, &a.geom};
    for (DevBuf *b : all) {
        cudaFree(b->p);
        b->p = nullptr;
        b->cap = 0;
    }
    for (int k = 0; k < 4; ++k) {
        for (DevBuf *b : {&a.lcnt[k], &a.loffs[k], &a.lids[k]}) {
            cudaFree(b->p);
            b->p = nullptr;
            b->cap = 0;
        }
    }
}

int evaluate_adaptive(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                      cudaStream_t s)
{
    AdaptiveState &A = ctx->ad;
    const int P = prm->p, PP = P * P;
    const int leaf_size = prm->leaf_size;
    const bool timing = (prm->flags & GBFMM_FLAG_STAGE_TIMING) != 0;
    auto mark = [&](int k) {
        if (timing) cudaEventRecord(ctx->ev[k], s);
    };
    const int64_t nblk = (n + 4095) / 4096;
    bool ok = true;
    auto need = [&](DevBuf &b, size_t bytes) {
        if (grow(b, bytes, false, 0, s) != 0) ok = false;
    };
    need(A.keys0, 8 * n);
    need(A.keys1, 8 * n);
    need(A.idx0, 4 * n);
    need(A.idx1, 4 * n);
    need(A.sx, 16 * n);
    need(A.far, 16 * n);
    need(A.hist, 4 * (256 * nblk + 1));
    need(A.scan_tmp, 4 * (exclusive_scan_tmp_words(n + 1) + exclusive_scan_tmp_words(256 * nblk) + 64));
    need(A.flags, 4 * (n + 1));
    need(A.scan, 4 * (n + 1));
    need(A.pcell, 4 * n);
    need(A.leaf_of, 4 * n);
    need(A.box, sizeof(Box));
    need(A.group_cnt, 4 * 2 * 8 * (kAdaptMaxLevel + 2));
    if (!ok) return fail(ctx, GBFMM_ENOMEM, "adaptive buffers");
    bool built_now = false;
    if (timing) cudaEventRecord(ctx->ev[kStages], s);
    int rc = ensure_ops(ctx, P, s, &built_now);
    if (rc != GBFMM_OK) return rc;
    const OpsCache &ops = ctx->ops[order_slot(P)];
    ctx->ops_built_last = built_now;

    // ---- box, keys, sort ----
    mark(0);
    const float4 *x = reinterpret_cast<const float4 *>(d_xyzq);
    Box *box = A.box.as<Box>();
    launch_bbox(x, n, prm->has_box, prm->box_origin, prm->box_side, box, ctx->d_partials, ctx->d_counter,
                ctx->d_status, s);
    k_keys64<<<blocks_for(n), 256, 0, s>>>(x, n, box, A.keys0.as<uint64_t>(), A.idx0.as<uint32_t>());
    note_launches(1);
    mark(1);
    uint64_t *skeys = nullptr;
    uint32_t *perm = nullptr;
    launch_sort_gather64(A.keys0.as<uint64_t>(), A.keys1.as<uint64_t>(), A.idx0.as<uint32_t>(),
                         A.idx1.as<uint32_t>(), n, 63, A.hist.as<uint32_t>(), nblk, A.scan_tmp.as<uint32_t>(), x,
                         A.sx.as<float4>(), &skeys, &perm, s);
    mark(2);

    // ---- tree, level by level ----
    int64_t cap = std::max<int64_t>(64, 2 * n / std::max(1, leaf_size) + 64);
    auto cell_bufs = [&](int64_t c, bool keep, int64_t used) {
        struct {
            DevBuf *b;
            size_t per;
        } cb[] = {{&A.level, 4}, {&A.key, 8}, {&A.begin, 4}, {&A.count, 4}, {&A.parent, 4}, {&A.child_begin, 4},
                  {&A.nchild, 4}, {&A.child_of, 32}};
        for (auto &e : cb)
            if (grow(*e.b, e.per * c, keep, e.per * used, s) != 0) return false;
        return true;
    };
    if (!cell_bufs(cap, false, 0)) return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
    k_tree_root<<<1, 1, 0, s>>>(n, A.level.as<int32_t>(), A.key.as<uint64_t>(), A.begin.as<int32_t>(),
                                A.count.as<int32_t>(), A.parent.as<int32_t>(), A.child_begin.as<int32_t>(),
                                A.nchild.as<int32_t>(), A.child_of.as<int32_t>());
    k_tree_pcell_init<<<blocks_for(n), 256, 0, s>>>(n, A.pcell.as<int32_t>());
    note_launches(2);
    std::vector<int> ls = {0, 1};
    int64_t ncells = 1;
    int maxl = 0;
    for (int l = 0; l < kAdaptMaxLevel + 1; ++l) {
        k_tree_flags<<<blocks_for(n), 256, 0, s>>>(n, skeys, l, leaf_size, kAdaptMaxLevel, A.pcell.as<int32_t>(),
                                                   A.count.as<int32_t>(), A.begin.as<int32_t>(),
                                                   A.flags.as<uint32_t>(), A.leaf_of.as<int32_t>());
        note_launches(1);
        launch_exclusive_scan(A.flags.as<uint32_t>(), A.scan.as<uint32_t>(), n, A.scan_tmp.as<uint32_t>(), s);
        const uint32_t nnew = read1<uint32_t>(A.scan.as<uint32_t>() + n, s);
        if (nnew == 0) break;
        if (ncells + nnew > cap) {
            int64_t ncap = std::max<int64_t>(2 * cap, ncells + nnew + 64);
            if (!cell_bufs(ncap, true, ncells)) return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
            cap = ncap;
        }
        k_tree_new_cells<<<blocks_for(n), 256, 0, s>>>(
            n, skeys, l, A.pcell.as<int32_t>(), A.flags.as<uint32_t>(), A.scan.as<uint32_t>(), ncells,
            A.level.as<int32_t>(), A.key.as<uint64_t>(), A.begin.as<int32_t>(), A.parent.as<int32_t>(),
            A.child_begin.as<int32_t>(), A.nchild.as<int32_t>(), A.child_of.as<int32_t>());
        k_tree_counts<<<blocks_for(nnew), 256, 0, s>>>(ncells, nnew, A.begin.as<int32_t>(), A.parent.as<int32_t>(),
                                                      A.count.as<int32_t>());
        k_tree_pcell<<<blocks_for(n), 256, 0, s>>>(n, A.flags.as<uint32_t>(), A.scan.as<uint32_t>(), ncells,
                                                  A.pcell.as<int32_t>());
        note_launches(3);
        ncells += nnew;
        ls.push_back((int)ncells);
        maxl = l + 1;
    }
    // particles still in a cell after the last level are in leaves of that level
    k_tree_flags<<<blocks_for(n), 256, 0, s>>>(n, skeys, kAdaptMaxLevel, leaf_size, kAdaptMaxLevel,
                                               A.pcell.as<int32_t>(), A.count.as<int32_t>(), A.begin.as<int32_t>(),
                                               A.flags.as<uint32_t>(), A.leaf_of.as<int32_t>());
    note_launches(1);
    A.ncells = ncells;
    A.max_level = maxl;
    A.level_start = ls;
    if (grow(A.end, 4 * ncells, false, 0, s) || grow(A.coll, 4 * 27 * ncells, false, 0, s) ||
        grow(A.leaves, 4 * ncells + 4, false, 0, s))
        return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
    k_cell_end<<<blocks_for(ncells), 256, 0, s>>>(ncells, A.begin.as<int32_t>(), A.count.as<int32_t>(),
                                                 A.end.as<int32_t>());
    note_launches(1);
    if (grow(A.geom, 16 * (size_t)ncells, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
    const float4 *geom = A.geom.as<float4>();
    launch_cell_geom(ncells, A.level.as<int32_t>(), A.key.as<uint64_t>(), box, A.geom.as<float4>(), s);
    for (int l = 0; l <= maxl; ++l) {
        const int64_t lo = ls[l], hi = ls[l + 1];
        k_colleagues<<<blocks_for(hi - lo), 256, 0, s>>>(lo, hi, l, A.key.as<uint64_t>(), A.parent.as<int32_t>(),
                                                        A.child_of.as<int32_t>(), A.coll.as<int32_t>());
        note_launches(1);
    }
    // leaf list
    cudaMemsetAsync(A.group_cnt.p, 0, A.group_cnt.cap, s);
    uint32_t *leaf_cursor = A.group_cnt.as<uint32_t>() + 8 * (kAdaptMaxLevel + 2) * 2 - 1;
    k_leaf_list<<<blocks_for(ncells), 256, 0, s>>>(ncells, A.nchild.as<int32_t>(), leaf_cursor,
                                                  A.leaves.as<int32_t>());
    note_launches(1);
    A.nleaves = read1<uint32_t>(leaf_cursor, s);

    // ---- lists ----
    if (grow(A.scan_tmp, 4 * (exclusive_scan_tmp_words(ncells + 1) + 64), false, 0, s))
        return fail(ctx, GBFMM_ENOMEM, "adaptive scan");
    TreeView tv{A.level.as<int32_t>(), A.parent.as<int32_t>(), A.nchild.as<int32_t>(), A.child_of.as<int32_t>(),
                A.coll.as<int32_t>(), A.key.as<uint64_t>()};
    for (int k = 0; k < 4; ++k) {
        if (grow(A.lcnt[k], 4 * (ncells + 1), false, 0, s) || grow(A.loffs[k], 4 * (ncells + 1), false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
        k_alist_count<<<blocks_for(ncells, 128), 128, 0, s>>>(k, ncells, tv, A.lcnt[k].as<uint32_t>(),
                                                             ctx->d_status);
        note_launches(1);
        launch_exclusive_scan(A.lcnt[k].as<uint32_t>(), A.loffs[k].as<uint32_t>(), ncells,
                              A.scan_tmp.as<uint32_t>(), s);
        const uint32_t ne = read1<uint32_t>(A.loffs[k].as<uint32_t>() + ncells, s);
        A.entries[k] = ne;
        if (grow(A.lids[k], 4 * (size_t)ne + 4, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
        if (k == kListV && grow(A.vcode, 2 * (size_t)ne + 4, false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
        k_alist_fill<<<blocks_for(ncells, 128), 128, 0, s>>>(k, ncells, tv, A.loffs[k].as<uint32_t>(),
                                                            A.lids[k].as<int32_t>(),
                                                            k == kListV ? A.vcode.as<uint16_t>() : nullptr);
        note_launches(1);
    }
    mark(3);

    // ---- expansions ----
    if (grow(A.M, 4 * (size_t)ncells * PP, false, 0, s) || grow(A.Lc, 4 * (size_t)ncells * PP, false, 0, s))
        return fail(ctx, GBFMM_ENOMEM, "adaptive expansions");
    float *M = A.M.as<float>(), *Lc = A.Lc.as<float>();
    float4 *far = A.far.as<float4>();
    const bool deep = maxl >= 2;
    if (deep) launch_p2m_cells(P, A.leaves.as<int32_t>(), A.nleaves, A.level.as<int32_t>(), geom,
                               A.begin.as<int32_t>(), A.count.as<int32_t>(), A.sx.as<float4>(), M, s);
    mark(4);
    for (int l = maxl - 1; l >= 2; --l)
        launch_translate_cells(P, true, ls[l], ls[l + 1] - ls[l], A.child_of.as<int32_t>(), A.nchild.as<int32_t>(),
                               ops.m2m, M, s);
    mark(5);
    if (deep) {
        // M2L targets: every cell at levels >= 2, grouped by (level, child position)
        const int64_t lo2 = ls[2];
        uint32_t *gcnt = A.group_cnt.as<uint32_t>();
        k_group_count<<<blocks_for(ncells - lo2), 256, 0, s>>>(lo2, ncells, A.level.as<int32_t>(),
                                                               A.key.as<uint64_t>(), gcnt);
        note_launches(1);
        std::vector<uint32_t> hcnt(8 * (kAdaptMaxLevel + 2));
        cudaMemcpyAsync(hcnt.data(), gcnt, 4 * hcnt.size(), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        std::vector<uint32_t> hcur(hcnt.size());
        std::vector<int4> tiles;
        const bool cores = (prm->flags & GBFMM_FLAG_M2L_CUDA_CORES) != 0;
        const bool f16 = ops.m2l_f16 != nullptr && !cores;
        const bool tc = f16 || (ops.m2l_tc != nullptr && !cores);
        const int TN = tc ? kM2LTcTargetsPerTile : kM2LTargetsPerTile;
        uint32_t acc = 0;
        for (int l = maxl; l >= 2; --l)
            for (int tau = 0; tau < 8; ++tau) {
                const int gi = l * 8 + tau;
                hcur[gi] = acc;
                for (uint32_t st = 0; st < hcnt[gi]; st += TN)
                    tiles.push_back(make_int4(l, tau, (int)(acc + st), (int)std::min<uint32_t>(TN, hcnt[gi] - st)));
                acc += hcnt[gi];
            }
        if (grow(A.tlist, 4 * (size_t)acc + 4, false, 0, s) || grow(A.tdesc, sizeof(int4) * tiles.size() + 16, false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive tiles");
        uint32_t *gcur = gcnt + 8 * (kAdaptMaxLevel + 2);
        cudaMemcpyAsync(gcur, hcur.data(), 4 * hcur.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(A.tdesc.p, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s);
        k_group_fill<<<blocks_for(ncells - lo2), 256, 0, s>>>(lo2, ncells, A.level.as<int32_t>(),
                                                              A.key.as<uint64_t>(), gcur, A.tlist.as<int32_t>());
        note_launches(1);
        cudaStreamSynchronize(s);  // the host tile vectors go out of scope
        if (f16) {
            if (grow(A.cscale, (size_t)ncells + 16, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive scales");
            launch_cell_scale(M, ncells, P, A.cscale.as<int8_t>(), s);
            launch_m2l_f16_tiles(P, A.tdesc.as<int4>(), (int)tiles.size(), A.tlist.as<int32_t>(), A.begin.as<int32_t>(),
                                 A.end.as<int32_t>(), A.loffs[kListV].as<uint32_t>(), A.lids[kListV].as<int32_t>(),
                                 A.vcode.as<uint16_t>(), ops.m2l_f16, M, A.cscale.as<int8_t>(), Lc, ctx->d_status, s);
        } else if (tc)
            launch_m2l_tc_tiles(P, A.tdesc.as<int4>(), (int)tiles.size(), A.tlist.as<int32_t>(), A.begin.as<int32_t>(),
                                A.end.as<int32_t>(), A.loffs[kListV].as<uint32_t>(), A.lids[kListV].as<int32_t>(),
                                A.vcode.as<uint16_t>(), ops.m2l_tc, M, Lc, ctx->d_status, s);
        else
            launch_m2l_tiles(P, A.tdesc.as<int4>(), (int)tiles.size(), A.tlist.as<int32_t>(), A.begin.as<int32_t>(),
                             A.end.as<int32_t>(), A.loffs[kListV].as<uint32_t>(), A.lids[kListV].as<int32_t>(),
                             A.vcode.as<uint16_t>(), ops.m2l, M, Lc, ctx->d_zero, ctx->d_status, s);
        launch_p2l_cells(P, ncells, A.level.as<int32_t>(), geom, A.begin.as<int32_t>(), A.count.as<int32_t>(),
                         A.loffs[kListX].as<uint32_t>(), A.lids[kListX].as<int32_t>(), A.sx.as<float4>(), Lc, s);
    }
    mark(6);
    for (int l = 3; l <= maxl; ++l)
        launch_translate_cells(P, false, ls[l - 1], ls[l] - ls[l - 1], A.child_of.as<int32_t>(),
                               A.nchild.as<int32_t>(), ops.l2l, Lc, s);
    mark(7);
    launch_l2p_cells(P, n, A.leaf_of.as<int32_t>(), A.level.as<int32_t>(), geom, A.sx.as<float4>(), Lc, far, s);
    if (deep)
        launch_m2p_cells(P, A.leaves.as<int32_t>(), A.nleaves, geom, A.begin.as<int32_t>(), A.count.as<int32_t>(),
                         A.loffs[kListW].as<uint32_t>(), A.lids[kListW].as<int32_t>(), A.sx.as<float4>(), M, far, s);
    mark(8);
    launch_p2p_cells(A.leaves.as<int32_t>(), A.nleaves, n, A.sx.as<float4>(), A.begin.as<int32_t>(),
                     A.end.as<int32_t>(), A.loffs[kListU].as<uint32_t>(), A.lids[kListU].as<int32_t>(), far, perm,
                     (float)prm->eps2, reinterpret_cast<float4 *>(d_out), s);
    mark(9);
    A.n = n;
    A.P = P;
    A.skeys = skeys;
    A.perm = perm;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adaptive launch");
    return GBFMM_OK;
}

int export_adaptive_tree(gbfmm_ctx *ctx, double *origin_side, int64_t *ncells, int32_t *level, uint64_t *key,
                         int32_t *begin, int32_t *count, int32_t *parent, uint32_t *perm)
{
    const AdaptiveState &A = ctx->ad;
    if (ncells) *ncells = A.ncells;
    const size_t nc = (size_t)A.ncells;
    if (origin_side) {
        Box b;
        cudaMemcpy(&b, A.box.p, sizeof(Box), cudaMemcpyDeviceToHost);
        for (int d = 0; d < 3; ++d) origin_side[d] = b.origin[d];
        origin_side[3] = b.side;
    }
    if (level) cudaMemcpy(level, A.level.p, 4 * nc, cudaMemcpyDeviceToHost);
    if (key) cudaMemcpy(key, A.key.p, 8 * nc, cudaMemcpyDeviceToHost);
    if (begin) cudaMemcpy(begin, A.begin.p, 4 * nc, cudaMemcpyDeviceToHost);
    if (count) cudaMemcpy(count, A.count.p, 4 * nc, cudaMemcpyDeviceToHost);
    if (parent) cudaMemcpy(parent, A.parent.p, 4 * nc, cudaMemcpyDeviceToHost);
    if (perm) cudaMemcpy(perm, A.perm, 4 * (size_t)A.n, cudaMemcpyDeviceToHost);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "export copy");
}

int export_adaptive_expansions(gbfmm_ctx *ctx, int which, double *coef)
{
    const AdaptiveState &A = ctx->ad;
    const int P = A.P, PP = P * P, NT = P * (P + 1) / 2;
    const size_t nc = (size_t)A.ncells;
    std::vector<float> v(nc * PP);
    std::vector<int32_t> lev(nc);
    Box box;
    cudaMemcpy(&box, A.box.p, sizeof(Box), cudaMemcpyDeviceToHost);
    if (A.max_level >= 2) cudaMemcpy(v.data(), which == 0 ? A.M.p : A.Lc.p, 4 * v.size(), cudaMemcpyDeviceToHost);
    cudaMemcpy(lev.data(), A.level.p, 4 * nc, cudaMemcpyDeviceToHost);
    for (size_t c = 0; c < nc; ++c) {
        const int l = lev[c];
        const double h = box.side / (double)(int64_t(1) << l);
        const bool formed = A.max_level >= 2 && l >= 2;
        double *out = coef + c * 2 * NT;
        for (int n = 0; n < P; ++n) {
            const double sc = which == 0 ? pow(h, n) : pow(h, -(n + 1));
            for (int m = 0; m <= n; ++m) {
                const int t = n * (n + 1) / 2 + m;
                double re = 0.0, im = 0.0;
                if (formed) {
                    const float *src = v.data() + c * PP;
                    re = src[m == 0 ? n * n : n * n + 2 * m - 1] * sc;
                    im = m == 0 ? 0.0 : src[n * n + 2 * m] * sc;
                }
                out[2 * t] = re;
                out[2 * t + 1] = im;
            }
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "export copy");
}

int export_adaptive_list(gbfmm_ctx *ctx, int kind, int32_t *offs, int32_t *ids, int64_t cap, int64_t *n_entries)
{
    const AdaptiveState &A = ctx->ad;
    const int64_t rows = A.ncells;
    std::vector<uint32_t> o(rows + 1);
    cudaMemcpy(o.data(), A.loffs[kind].p, 4 * (rows + 1), cudaMemcpyDeviceToHost);
    const int64_t ne = o[rows];
    if (n_entries) *n_entries = ne;
    if (offs)
        for (int64_t r = 0; r <= rows; ++r) offs[r] = (int32_t)o[r];
    if (ids) {
        if (cap < ne) return fail(ctx, GBFMM_ENOMEM, "ids capacity too small");
        cudaMemcpy(ids, A.lids[kind].p, 4 * ne, cudaMemcpyDeviceToHost);
        for (int64_t r = 0; r < rows; ++r) std::sort(ids + o[r], ids + o[r + 1]);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBFMM_OK : cuda_fail(ctx, e, "export copy");
}

}  // namespace gbfmm
