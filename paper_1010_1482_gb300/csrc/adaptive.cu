// Adaptive octree FMM on the device (the adaptive FMM of Cheng, Greengard & Rokhlin 1999,
// which the paper cites for its translation operators).
//
// Tree: the particles are sorted by their full 63-bit Morton key (stable radix sort); a cell
// splits while it holds more than leaf_size particles (and is above level 21); only nonempty
// children exist.  Cells are numbered level by level, in key order within a level.  The cells
// are found in one pass over the sorted keys (every particle learns the levels at which it
// starts a cell); leaf sizes beyond the one-pass window take level-by-level rounds.
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
constexpr int64_t kListWarpCells = 1 << 17;  // below this many cells the U/W/X rows take a warp per cell

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
    for (int d = 0; d < 3; ++d) k[d] = grid_coord21(c[d], b, d);  // the FP64 steps' result
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

// ---- one-pass construction ------------------------------------------------------------------
// With the particles sorted by key, let cpl(a, b) be the deepest level d at which keys a and b
// have the same level-d prefix (21 for equal keys).  For a window of leaf_size + 1 consecutive
// particles j..j+leaf_size, w_j = cpl(key_j, key_{j+leaf_size}) is the deepest level whose cell
// holds the whole window.  The level-d cell of particle i holds more than leaf_size particles
// exactly when some window containing i lies inside it, so
//   D_i = max over j in [i - leaf_size, i] of w_j      (-1 if no window fits in [0, n))
// is the deepest level at which i's cell would split by count, and i's leaf is at level
//   lambda_i = D_i < 0 ? 0 : min(D_i, 20) + 1.
// Particle i is the first particle of its level-l cell for l >= a_i = cpl(key_{i-1}, key_i) + 1
// (a_0 = 0), and that cell exists when l <= lambda_i (every ancestor splits).  So i starts the
// cells of levels a_i..lambda_i, and the cells of level l, numbered level by level in key
// order, are ranked by a per-level count over the particles: the same cells, numbering and
// fields as the level-by-level rounds, with one host read (the level sizes) instead of one
// per level.
constexpr int kTreeB = 256;                      // particles per block
constexpr int kTreeBins = kAdaptMaxLevel + 2;    // levels 0..21, then leaf starts
constexpr int kTreeMaxWindow = 16384;            // leaf sizes above this take the level rounds

GB_DEV int cpl63(uint64_t a, uint64_t b)
{
    const uint64_t x = a ^ b;
    if (x == 0) return kAdaptMaxLevel;
    return kAdaptMaxLevel - 1 - (63 - __clzll((long long)x)) / 3;
}

GB_DEV bool tree_bin(int bin, int a, int lam) { return bin < kTreeBins - 1 ? (a <= bin && bin <= lam) : (a <= lam); }

// per particle: (a_i, lambda_i) packed as a | lambda << 8, and per block the count of each bin;
// the window maxima come from a sparse table in shared memory over w_j, j in [i0 - leaf, i0 + B)
__global__ void __launch_bounds__(kTreeB) k_tree_ranges(int64_t n, const uint64_t *__restrict__ sk, int leaf,
                                                        int64_t nblk, uint16_t *__restrict__ range,
                                                        uint32_t *__restrict__ hist)
{
    extern __shared__ int8_t wbuf[];  // 2 (B + leaf): ping-pong
    __shared__ uint32_t wc[kTreeB / 32][kTreeBins];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = blockIdx.x * (int64_t)kTreeB;
    const int size = kTreeB + leaf;
    int8_t *src = wbuf, *dst = wbuf + size;
    for (int jj = tid; jj < size; jj += kTreeB) {
        const int64_t j = i0 - leaf + jj;
        int w = -1;
        if (j >= 0 && j + leaf < n) w = cpl63(sk[j], sk[j + leaf]);
        src[jj] = (int8_t)w;
    }
    __syncthreads();
    int k = 0;
    while ((2 << k) <= leaf + 1) ++k;  // 2^k <= leaf + 1 < 2^(k+1)
    for (int t = 0; t < k; ++t) {
        const int d = 1 << t;
        for (int jj = tid; jj < size; jj += kTreeB) {
            int8_t v = src[jj];
            if (jj + d < size) v = max(v, src[jj + d]);
            dst[jj] = v;
        }
        __syncthreads();
        int8_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    const int64_t i = i0 + tid;
    int a = kAdaptMaxLevel + 1, lam = -1;
    if (i < n) {
        const int dm = max((int)src[tid], (int)src[tid + leaf + 1 - (1 << k)]);
        lam = dm < 0 ? 0 : min(dm, kAdaptMaxLevel - 1) + 1;
        a = i == 0 ? 0 : cpl63(sk[i - 1], sk[i]) + 1;
        range[i] = (uint16_t)(a | (lam << 8));
    }
    for (int b = 0; b < kTreeBins; ++b) {
        const unsigned bal = __ballot_sync(0xffffffffu, tree_bin(b, a, lam));
        if (lane == 0) wc[warp][b] = __popc(bal);
    }
    __syncthreads();
    if (tid < kTreeBins) {
        uint32_t sum = 0;
        for (int w = 0; w < kTreeB / 32; ++w) sum += wc[w][tid];
        hist[(int64_t)tid * nblk + blockIdx.x] = sum;
    }
}

// info[b] = first index of bin b (level starts, then the number of cells), info[kTreeBins] =
// cells + leaves
__global__ void k_tree_starts(int64_t nblk, const uint32_t *__restrict__ base, int32_t *__restrict__ info)
{
    const int t = threadIdx.x;
    if (t <= kTreeBins) info[t] = (int32_t)base[(int64_t)t * nblk];
}

// writes every cell a particle starts (level, key, begin, parent when it starts there too),
// the leaf list in key order and every particle's leaf ordinal (into leaf_ord)
__global__ void __launch_bounds__(kTreeB) k_tree_cells(int64_t n, const uint64_t *__restrict__ sk, int64_t nblk,
                                                       const uint16_t *__restrict__ range,
                                                       const uint32_t *__restrict__ base, int32_t *__restrict__ level,
                                                       uint64_t *__restrict__ key, int32_t *__restrict__ begin,
                                                       int32_t *__restrict__ parent, int32_t *__restrict__ child_begin,
                                                       int32_t *__restrict__ nchild, int32_t *__restrict__ child_of,
                                                       int32_t *__restrict__ leaves, int32_t *__restrict__ leaf_ord,
                                                       const int32_t *__restrict__ abort)
{
    __shared__ uint32_t wc[kTreeB / 32][kTreeBins];
    __shared__ uint32_t sb0[kTreeBins], sbl;
    if (abort && *abort) return;  // the tree outgrew the capacities: nothing is written
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = blockIdx.x * (int64_t)kTreeB + tid;
    int a = kAdaptMaxLevel + 1, lam = -1;
    uint64_t kk = 0;
    if (i < n) {
        const uint16_t r = range[i];
        a = r & 0xff;
        lam = r >> 8;
        kk = sk[i];
    }
    for (int b = 0; b < kTreeBins; ++b) {
        const unsigned bal = __ballot_sync(0xffffffffu, tree_bin(b, a, lam));
        if (lane == 0) wc[warp][b] = __popc(bal);
    }
    __syncthreads();
    // per bin: the warps' counts become their exclusive offsets; the block's first index and
    // (leaves) the first leaf index, from the scanned histogram
    if (tid < kTreeBins) {
        uint32_t acc = 0;
        for (int w = 0; w < kTreeB / 32; ++w) {
            const uint32_t t = wc[w][tid];
            wc[w][tid] = acc;
            acc += t;
        }
        sb0[tid] = base[(int64_t)tid * nblk + blockIdx.x];
        if (tid == kTreeBins - 1) sbl = base[(int64_t)tid * nblk];
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int32_t prev = -1;
#pragma unroll
    for (int b = 0; b < kTreeBins; ++b) {
        const bool p = tree_bin(b, a, lam);
        const unsigned bal = __ballot_sync(0xffffffffu, p);
        const uint32_t off = __popc(bal & lt) + wc[warp][b];
        const uint32_t b0 = sb0[b];
        if (b < kTreeBins - 1) {
            if (!p) continue;
            const int32_t id = (int32_t)(b0 + off);
            level[id] = b;
            key[id] = kk >> (3 * (kAdaptMaxLevel - b));
            begin[id] = (int32_t)i;
            parent[id] = b == 0 ? -1 : (b > a ? prev : -2);
            child_begin[id] = 0x7fffffff;
            nchild[id] = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) child_of[(int64_t)id * 8 + q] = -1;
            prev = id;
        } else if (i < n) {
            const int64_t ord = (int64_t)b0 - (int64_t)sbl + off + (p ? 1 : 0) - 1;
            leaf_ord[i] = (int32_t)ord;
            if (p) leaves[ord] = prev;  // the cell of level lambda_i
        }
    }
}

// per cell: particle count (end of its key prefix in the sorted keys), the parent of a cell
// whose parent starts at an earlier particle (key search within the parent level), and the
// parent's child links
__global__ void k_tree_links(Span cells, int64_t n, const uint64_t *__restrict__ sk, const int32_t *__restrict__ info,
                             const int32_t *__restrict__ level, const uint64_t *__restrict__ key,
                             const int32_t *__restrict__ begin, int32_t *__restrict__ count, int32_t *__restrict__ end,
                             int32_t *__restrict__ parent, int32_t *__restrict__ child_begin,
                             int32_t *__restrict__ nchild, int32_t *__restrict__ child_of)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
    const int l = level[c];
    const uint64_t kk = key[c];
    const int64_t b = begin[c];
    int64_t e = n;
    if (l > 0) {
        const int sh = 3 * (kAdaptMaxLevel - l);
        int64_t lo = b + 1, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((sk[mid] >> sh) == kk)
                lo = mid + 1;
            else
                hi = mid;
        }
        e = lo;
    }
    count[c] = (int32_t)(e - b);
    end[c] = (int32_t)e;
    int32_t p = parent[c];
    if (p == -2) {
        const uint64_t pk = kk >> 3;
        int32_t lo = info[l - 1], hi = info[l] - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (key[mid] < pk)
                lo = mid + 1;
            else
                hi = mid;
        }
        p = lo;
        parent[c] = p;
    }
    if (p >= 0) {
        child_of[(int64_t)p * 8 + (int)(kk & 7)] = (int32_t)c;
        atomicAdd(&nchild[p], 1);
        atomicMin(&child_begin[p], (int32_t)c);
    }
}

__global__ void k_tree_leaf_of(int64_t n, const int32_t *__restrict__ leaves, int32_t *__restrict__ leaf_of,
                               const int32_t *__restrict__ abort)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !(abort && *abort)) leaf_of[i] = leaves[leaf_of[i]];
}

// list sizes of the four kinds into info[0..3]
__global__ void k_list_totals(int64_t nc, const uint32_t *o0, const uint32_t *o1, const uint32_t *o2,
                              const uint32_t *o3, int32_t *info)
{
    if (threadIdx.x == 0) {
        info[0] = (int32_t)o0[nc];
        info[1] = (int32_t)o1[nc];
        info[2] = (int32_t)o2[nc];
        info[3] = (int32_t)o3[nc];
    }
}

__global__ void k_cell_end(int64_t nc, const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                           int32_t *__restrict__ end)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < nc) end[c] = begin[c] + count[c];
}

// ---- colleagues (positional: slot (dx+1) + 3(dy+1) + 9(dz+1)) -----------------------------
GB_DEV int slot27(int dx, int dy, int dz) { return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1); }

__global__ void k_colleagues(Span lv, int l, const uint64_t *__restrict__ key, const int32_t *__restrict__ parent,
                             const int32_t *__restrict__ child_of, int32_t *__restrict__ coll)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(lv)) return;
    const int64_t b = span_first(lv) + i;
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
    const int4 *anc;  // integer box at depth 21: anchor x, y, z and log2 of the side
};

// integer box of every cell at depth 21 (the adjacency tests read it instead of decoding keys)
__global__ void k_cell_anchor(Span cells, const int32_t *__restrict__ level, const uint64_t *__restrict__ key,
                              int4 *__restrict__ anc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
    int x, y, z;
    demorton63(key[c], x, y, z);
    const int sh = kAdaptMaxLevel - level[c];
    anc[c] = make_int4(x << sh, y << sh, z << sh, sh);
}

// boxes that touch or overlap in all three dimensions
GB_DEV bool adjacent(const TreeView &t, int32_t a, int32_t b)
{
    const int4 la = t.anc[a], lb = t.anc[b];
    const int sa = 1 << la.w, sb = 1 << lb.w;
    return !(la.x > lb.x + sb || lb.x > la.x + sa || la.y > lb.y + sb || lb.y > la.y + sa || la.z > lb.z + sb ||
             lb.z > la.z + sa);
}

// Descent below colleague a of leaf b (U and W lists): a leaf colleague is a U entry; below a
// split colleague, descendants adjacent to b are opened (leaves among them are U entries) and
// the first non-adjacent ones on each path are W entries.  Calls f(id) for the entries of the
// list kind; returns false if the stack overflowed.
template <bool U, class F>
GB_DEV bool descend(const TreeView &t, int32_t b, int32_t a, F f)
{
    if (a < 0) return true;
    if (t.nchild[a] == 0) {
        if (U) f(a);
        return true;
    }
    bool ok = true;
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
                if (U) f(d);
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
        } else if (!U) {
            f(d);
        }
    }
    return ok;
}

GB_DEV uint32_t warp_excl_scan(uint32_t v, int lane, uint32_t &total)
{
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// U, W and X lists, one warp per cell.  Entries come in the order: colleague slot (lane), the
// descent below it, then (U, X) ancestors from the parent up, colleague slot within each.  The
// count pass (FILL = false) writes the row lengths; the fill pass writes the rows at `offs`.
template <int KIND, bool FILL>
__global__ void k_alist_warp(Span cells, TreeView t, uint32_t *__restrict__ cnt, const uint32_t *__restrict__ offs,
                             int32_t *__restrict__ ids, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= span_count(cells)) return;
    const int64_t bb = span_first(cells) + w;
    const int32_t b = (int32_t)bb;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t e = FILL ? offs[b] : 0u;
    if (KIND == kListU || KIND == kListW) {
        if (t.nchild[b] != 0) {
            if (!FILL && lane == 0) cnt[b] = 0;
            return;
        }
        const int32_t a = lane < 27 ? t.coll[(int64_t)b * 27 + lane] : -1;
        uint32_t mine = 0;
        const bool ok = descend<KIND == kListU>(t, b, a, [&](int32_t) { ++mine; });
        if (!FILL && !ok) atomicOr(status, kStatusTimeout);
        uint32_t total;
        const uint32_t excl = warp_excl_scan(mine, lane, total);
        if (FILL) {
            uint32_t w = e + excl;
            descend<KIND == kListU>(t, b, a, [&](int32_t d) { ids[w++] = d; });
        }
        e += total;
    }
    if (KIND == kListU || KIND == kListX) {
        const int32_t ref = KIND == kListU ? b : t.parent[b];  // adjacency reference
        if (ref >= 0)
            for (int32_t anc = t.parent[b]; anc >= 0; anc = t.parent[anc]) {
                const int32_t c = lane < 27 ? t.coll[(int64_t)anc * 27 + lane] : -1;
                bool hit = c >= 0 && c != anc && t.nchild[c] == 0 && adjacent(t, ref, c);
                if (KIND == kListX && hit) hit = !adjacent(t, b, c);
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (FILL && hit) ids[e + __popc(bal & lt)] = c;
                e += __popc(bal);
            }
    }
    if (!FILL && lane == 0) cnt[b] = e;
}

// The same U, W and X rows, one thread per cell (slots in sequence): on large trees the warp
// form leaves most lanes idle while one descends, and its fill repeats the descents.
template <int KIND, bool FILL>
__global__ void k_alist_thread(Span cells, TreeView t, uint32_t *__restrict__ cnt, const uint32_t *__restrict__ offs,
                               int32_t *__restrict__ ids, int *status)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t bb = span_first(cells) + i;
    const int32_t b = (int32_t)bb;
    uint32_t e = FILL ? offs[b] : 0u;
    auto emit = [&](int32_t d) {
        if (FILL) ids[e] = d;
        ++e;
    };
    if (KIND == kListU || KIND == kListW) {
        if (t.nchild[b] != 0) {
            if (!FILL) cnt[b] = 0;
            return;
        }
        bool ok = true;
        for (int sl = 0; sl < 27; ++sl) ok &= descend<KIND == kListU>(t, b, t.coll[(int64_t)b * 27 + sl], emit);
        if (!FILL && !ok) atomicOr(status, kStatusTimeout);
    }
    if (KIND == kListU || KIND == kListX) {
        const int32_t ref = KIND == kListU ? b : t.parent[b];
        if (ref >= 0)
            for (int32_t anc = t.parent[b]; anc >= 0; anc = t.parent[anc])
                for (int sl = 0; sl < 27; ++sl) {
                    const int32_t c = t.coll[(int64_t)anc * 27 + sl];
                    if (c < 0 || c == anc || t.nchild[c] != 0 || !adjacent(t, ref, c)) continue;
                    if (KIND == kListX && adjacent(t, b, c)) continue;
                    emit(c);
                }
    }
    if (!FILL) cnt[b] = e;
}

// V list, one warp per cell: lane j takes the candidate offsets t = j, j + 32, ... of the
// 6x6x6 block of the parent's colleagues' children (t = 36 (oz + 2 + cz) + 6 (oy + 2 + cy) +
// (ox + 2 + cx): oz slowest, ox fastest), and a ballot compacts the hits so that a row is
// written in that order with coalesced stores.
template <bool FILL>
__global__ void k_vlist_warp(Span cells, TreeView t, uint32_t *__restrict__ cnt, const uint32_t *__restrict__ offs,
                             int32_t *__restrict__ ids, uint16_t *__restrict__ codes)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= span_count(cells)) return;
    const int64_t b = span_first(cells) + w;
    const int l = t.level[b];
    if (l < 2) {
        if (!FILL && lane == 0) cnt[b] = 0;
        return;
    }
    int x, y, z;
    demorton63(t.key[b], x, y, z);
    const int side = 1 << l, cx = x & 1, cy = y & 1, cz = z & 1;
    // the parent's 27 colleagues, one per lane, read once per cell and shuffled to the candidates
    const int32_t pcv = lane < 27 ? t.coll[(int64_t)t.parent[b] * 27 + lane] : -1;
    uint32_t e = FILL ? offs[b] : 0u;
    for (int t0 = 0; t0 < 216; t0 += 32) {
        const int u = t0 + lane;
        const int ox = u % 6 - 2 - cx, oy = (u / 6) % 6 - 2 - cy, oz = u / 36 - 2 - cz;
        const int nx = x + ox, ny = y + oy, nz = z + oz;
        const bool cand = u < 216 && !(ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) &&
                          nx >= 0 && ny >= 0 && nz >= 0 && nx < side && ny < side && nz < side;
        const int sl = cand ? slot27((nx >> 1) - (x >> 1), (ny >> 1) - (y >> 1), (nz >> 1) - (z >> 1)) : 13;
        const int32_t a = __shfl_sync(0xffffffffu, pcv, sl);
        int32_t src = -1;
        if (cand && a >= 0) src = t.child_of[(int64_t)a * 8 + ((nx & 1) | ((ny & 1) << 1) | ((nz & 1) << 2))];
        const unsigned hit = __ballot_sync(0xffffffffu, src >= 0);
        if (FILL && src >= 0) {
            const uint32_t at = e + __popc(hit & ((1u << lane) - 1u));
            ids[at] = src;
            codes[at] = (uint16_t)m2l_code(ox, oy, oz);
        }
        e += __popc(hit);
    }
    if (!FILL && lane == 0) cnt[b] = e;
}

// ---- M2L targets grouped by (level, child position) ----------------------------------------
__global__ void k_group_count(Span cells, const int32_t *__restrict__ level, const uint64_t *__restrict__ key,
                              uint32_t *__restrict__ gcnt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
    atomicAdd(&gcnt[level[c] * 8 + (int)(key[c] & 7)], 1u);
}

__global__ void k_group_fill(Span cells, const int32_t *__restrict__ level, const uint64_t *__restrict__ key,
                             uint32_t *__restrict__ gcur, int32_t *__restrict__ tlist)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
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

// Treecode lists of a leaf B: its own row of list A followed by the rows of list B of B and of
// each ancestor up to the root (W then V for M2P; U then X for P2P).  Cells with children
// get empty rows.  The ancestor walk stops after kAdaptMaxLevel + 1 cells whatever the links.
__global__ void k_chain_count(Span cells, const int32_t *__restrict__ nchild, const int32_t *__restrict__ parent,
                              const uint32_t *__restrict__ offs_a, const uint32_t *__restrict__ offs_b,
                              uint32_t *__restrict__ cnt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
    uint32_t k = 0;
    if (nchild[c] == 0) {
        k = offs_a[c + 1] - offs_a[c];
        int32_t a = (int32_t)c;
        for (int d = 0; d <= kAdaptMaxLevel && a >= 0; ++d, a = parent[a]) k += offs_b[a + 1] - offs_b[a];
    }
    cnt[c] = k;
}

// a warp per leaf copies the rows counted by k_chain_count into its slice of ids
__global__ void k_chain_fill(Span cells, const int32_t *__restrict__ nchild, const int32_t *__restrict__ parent,
                             const uint32_t *__restrict__ offs_a, const int32_t *__restrict__ ids_a,
                             const uint32_t *__restrict__ offs_b, const int32_t *__restrict__ ids_b,
                             const uint32_t *__restrict__ offs, int32_t *__restrict__ ids)
{
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= span_count(cells)) return;
    const int64_t c = span_first(cells) + w;
    if (nchild[c] != 0) return;
    uint32_t o = offs[c];
    const uint32_t o_end = offs[c + 1];
    auto copy = [&](const int32_t *src, uint32_t e0, uint32_t e1) {
        for (uint32_t e = e0 + lane; e < e1; e += 32)
            if (o + (e - e0) < o_end) ids[o + (e - e0)] = src[e];
        o += e1 - e0;
    };
    copy(ids_a, offs_a[c], offs_a[c + 1]);
    int32_t a = (int32_t)c;
    for (int d = 0; d <= kAdaptMaxLevel && a >= 0; ++d, a = parent[a]) copy(ids_b, offs_b[a], offs_b[a + 1]);
}

// ---- capacities of captured evaluations --------------------------------------------------------
// info words: [0, kTreeBins] level starts, cells and cells + leaves (k_tree_starts); [32, 36) the
// list totals; [40, 42) the treecode chain totals; kInfoAbort: set when a count exceeds its
// capacity, after which every remaining launch of the evaluation does nothing
constexpr int kInfoLists = 32, kInfoChain = 40, kInfoAbort = 48;

struct GuardCaps {
    int64_t v[kTreeBins + 1];
};

// stage 0: the tree (cells, leaves, the cells of every level); stage 1: the four lists;
// stage 2: the chain lists.  A count above its capacity sets the abort word and kStatusCapacity.
__global__ void k_guard(const int32_t *__restrict__ info, GuardCaps g, int stage, int32_t *__restrict__ abort,
                        int *__restrict__ status)
{
    if (threadIdx.x != 0) return;
    bool over = false;
    if (stage == 0) {
        over = info[kTreeBins - 1] > g.v[0] || info[kTreeBins] - info[kTreeBins - 1] > g.v[1];
        for (int l = 0; l <= kAdaptMaxLevel; ++l) over = over || (info[l + 1] - info[l] > g.v[2 + l]);
    } else {
        const int base = stage == 1 ? kInfoLists : kInfoChain, k = stage == 1 ? 4 : 2;
        for (int j = 0; j < k; ++j) over = over || info[base + j] > g.v[j];
    }
    if (over) {
        *abort = 1;
        atomicOr(status, kStatusCapacity);
    }
}

// M2L tiles from the per-(level, child position) target counts, in the order levels 21 .. 2,
// child positions 0 .. 7, TN targets per tile: gcur[g] = the first tlist slot of group g, and
// tdesc[t] = (level, position, first slot, count) for t < tcap, count 0 past the last tile (or
// for every tile once the evaluation is aborted).  One CTA.
__global__ void k_tile_plan(const uint32_t *__restrict__ gcnt, uint32_t *__restrict__ gcur, int4 *__restrict__ tdesc,
                            int64_t tcap, int TN, const int32_t *__restrict__ abort)
{
    constexpr int NG = 8 * (kAdaptMaxLevel + 1);
    __shared__ uint32_t s_t0[NG + 1], s_slot[NG];
    __shared__ int s_g[NG];
    if (threadIdx.x == 0) {
        const bool ab = abort && *abort;
        uint32_t slot = 0, t = 0;
        int k = 0;
        for (int l = kAdaptMaxLevel; l >= 2; --l)
            for (int tau = 0; tau < 8; ++tau) {
                const int g = l * 8 + tau;
                const uint32_t c = ab ? 0u : gcnt[g];
                gcur[g] = slot;
                s_g[k] = g;
                s_slot[k] = slot;
                s_t0[k] = t;
                ++k;
                slot += c;
                t += (c + TN - 1) / TN;
            }
        s_t0[k] = t;
        s_g[k] = -1;
    }
    __syncthreads();
    const int ng = 8 * (kAdaptMaxLevel - 1);
    for (int64_t t = threadIdx.x; t < tcap; t += blockDim.x) {
        int4 d = make_int4(0, 0, 0, 0);
        if (t < s_t0[ng]) {
            int lo = 0, hi = ng - 1;  // the group k with s_t0[k] <= t < s_t0[k + 1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_t0[mid] <= t)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const int g = s_g[lo];
            const uint32_t j = (uint32_t)(t - s_t0[lo]) * TN;
            const uint32_t c = gcnt[g];
            d = make_int4(g / 8, g % 8, (int)(s_slot[lo] + j), (int)min((uint32_t)TN, c - j));
        }
        tdesc[t] = d;
    }
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
                     &a.leaves, &a.group_cnt, &a.cscale, &a.geom, &a.info, &a.anchor, &a.presplit, &a.near,
                     &a.tc_cnt, &a.tc_offs[0], &a.tc_offs[1], &a.tc_ids[0], &a.tc_ids[1], &a.partials,
                     &a.ab_flag, &a.ab_scan, &a.ab_unit_of, &a.ab_units, &a.ab_nu, &a.ab_pre, &a.ab_scale,
                     &a.ab_src, &a.lpart};
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

namespace {

// Launch ranges of one evaluation: from counts the host read back (exact sizes), or, under
// capacities, read on the device (cells: ncells capacity; levels: the per-level capacities).
struct Ranges {
    bool dev = false;
    const int32_t *info = nullptr, *abort = nullptr;
    int64_t ncells = 0, nleaves = 0;
    const std::vector<int> *ls = nullptr;
    const AdaptCaps *caps = nullptr;
    Span cells() const { return dev ? Span{0, ncells, nullptr, info + kTreeBins - 1, abort} : host_span(0, ncells); }
    // leaf ordinals (a span over the leaf list)
    Span leaves() const
    {
        return dev ? Span{0, nleaves, info + kTreeBins - 1, info + kTreeBins, abort} : host_span(0, nleaves);
    }
    Span level(int l) const
    {
        return dev ? Span{0, caps->level[l], info + l, info + l + 1, abort}
                   : host_span((*ls)[l], (*ls)[l + 1] - (*ls)[l]);
    }
    // the cells of levels >= 2
    Span deep() const
    {
        return dev ? Span{0, ncells, info + 2, info + kTreeBins - 1, abort} : host_span((*ls)[2], ncells - (*ls)[2]);
    }
};

// The treecode on the adaptive tree, once the tree and its U, V, W, X lists are built: P2M at
// the leaves and M2M up to level 2, then per leaf M2P over W and the ancestors' V rows and P2P
// over U and the ancestors' X rows, the M2P sums added in P2P's epilogue.  No local expansions.
template <class Mark>
int treecode_adaptive(gbfmm_ctx *ctx, AdaptiveState &A, const Ranges &R, const gbfmm_params *prm, int64_t n,
                      float *d_out, cudaStream_t s, Mark &mark)
{
    const int P = prm->p, PP = P * P;
    const int64_t ncells = R.ncells;
    const int maxl = A.max_level;
    const OpsCache &ops = ctx->ops[order_slot(P)];
    ctx->stage_order_last = 0;
    // chain lists: [0] U + ancestors' X (P2P), [1] W + ancestors' V (M2P)
    if (grow(A.tc_cnt, 4 * (ncells + 1), false, 0, s) || grow(A.tc_offs[0], 4 * (ncells + 1), false, 0, s) ||
        grow(A.tc_offs[1], 4 * (ncells + 1), false, 0, s))
        return fail(ctx, GBFMM_ENOMEM, "treecode lists");
    const int ka[2] = {kListU, kListW}, kb[2] = {kListX, kListV};
    for (int j = 0; j < 2; ++j) {
        if (R.dev) cudaMemsetAsync(A.tc_cnt.p, 0, 4 * (ncells + 1), s);
        k_chain_count<<<blocks_for(ncells), 256, 0, s>>>(R.cells(), A.nchild.as<int32_t>(), A.parent.as<int32_t>(),
                                                         A.loffs[ka[j]].as<uint32_t>(), A.loffs[kb[j]].as<uint32_t>(),
                                                         A.tc_cnt.as<uint32_t>());
        note_launches(1);
        launch_exclusive_scan(A.tc_cnt.as<uint32_t>(), A.tc_offs[j].as<uint32_t>(), ncells, A.scan_tmp.as<uint32_t>(),
                              s);
    }
    int32_t *info = A.info.as<int32_t>();
    k_list_totals<<<1, 32, 0, s>>>(ncells, A.tc_offs[0].as<uint32_t>(), A.tc_offs[1].as<uint32_t>(),
                                   A.tc_offs[0].as<uint32_t>(), A.tc_offs[1].as<uint32_t>(), info + kInfoChain);
    note_launches(1);
    int64_t tot[2];
    if (!R.dev) {
        int32_t h[4];
        cudaMemcpyAsync(h, info + kInfoChain, sizeof(h), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        for (int j = 0; j < 2; ++j) A.counts.chain[j] = tot[j] = (uint32_t)h[j];
    } else {
        GuardCaps g{};
        for (int j = 0; j < 2; ++j) g.v[j] = tot[j] = R.caps->chain[j];
        k_guard<<<1, 32, 0, s>>>(info, g, 2, info + kInfoAbort, ctx->d_status);
        note_launches(1);
    }
    for (int j = 0; j < 2; ++j) {
        if (grow(A.tc_ids[j], 4 * (size_t)tot[j] + 4, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "treecode lists");
        k_chain_fill<<<blocks_for(ncells, 8), 256, 0, s>>>(
            R.cells(), A.nchild.as<int32_t>(), A.parent.as<int32_t>(), A.loffs[ka[j]].as<uint32_t>(),
            A.lids[ka[j]].as<int32_t>(), A.loffs[kb[j]].as<uint32_t>(), A.lids[kb[j]].as<int32_t>(),
            A.tc_offs[j].as<uint32_t>(), A.tc_ids[j].as<int32_t>());
        note_launches(1);
    }

    if (grow(A.M, 4 * (size_t)ncells * PP, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive expansions");
    float *M = A.M.as<float>();
    float4 *far = A.far.as<float4>();
    const float4 *geom = A.geom.as<float4>();
    const bool deep = maxl >= 2;
    if (deep) launch_p2m_cells(P, A.leaves.as<int32_t>(), R.leaves(), A.level.as<int32_t>(), geom,
                               A.begin.as<int32_t>(), A.count.as<int32_t>(), A.sx.as<float4>(), M, s);
    mark(4);
    for (int l = maxl - 1; l >= 2; --l)
        launch_translate_cells(P, true, R.level(l), A.child_of.as<int32_t>(), A.nchild.as<int32_t>(), ops.m2m, M, s);
    mark(5);
    cudaMemsetAsync(far, 0, 16 * (size_t)n, s);
    if (deep)
        launch_m2p_cells(P, A.leaves.as<int32_t>(), R.leaves(), geom, A.begin.as<int32_t>(), A.end.as<int32_t>(),
                         A.tc_offs[1].as<uint32_t>(), A.tc_ids[1].as<int32_t>(), A.sx.as<float4>(), M, far, s,
                         true);
    mark(6);  // M2P is reported with M2L; no L2L, no L2P
    mark(7);
    mark(8);
    launch_p2p_cells(A.leaves.as<int32_t>(), R.leaves(), n, A.sx.as<float4>(), A.begin.as<int32_t>(),
                     A.end.as<int32_t>(), A.tc_offs[0].as<uint32_t>(), A.tc_ids[0].as<int32_t>(), far, A.perm,
                     (float)prm->eps2, reinterpret_cast<float4 *>(d_out), ctx->d_status, s);
    mark(9);
    A.P = P;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adaptive treecode launch");
    return GBFMM_OK;
}

}  // namespace

int evaluate_adaptive(gbfmm_ctx *ctx, const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_out,
                      cudaStream_t s)
{
    return evaluate_adaptive_in(ctx, ctx->ad, nullptr, prm, n, d_xyzq, d_out, s, ctx->d_partials, ctx->d_counter);
}

int evaluate_adaptive_in(gbfmm_ctx *ctx, AdaptiveState &A, const AdaptCaps *caps, const gbfmm_params *prm,
                         int64_t n, const float *d_xyzq, float *d_out, cudaStream_t s, float *partials,
                         unsigned *counter)
{
    set_p2p_leaves_per_cta(ctx->p2p_leaves_per_cta);
    const bool dev = caps != nullptr;
    const int P = prm->p, PP = P * P;
    const int leaf_size = prm->leaf_size;
    const bool timing = !dev && (prm->flags & GBFMM_FLAG_STAGE_TIMING) != 0;
    auto mark = [&](int k) {
        if (timing) cudaEventRecord(ctx->ev[k], s);
    };
    const int64_t window = std::min<int64_t>(leaf_size, n);
    if (dev && !caps->valid) return fail(ctx, GBFMM_EINVAL, "adaptive capacities not set");
    if (dev && !(n > 0 && window <= kTreeMaxWindow))
        return fail(ctx, GBFMM_EUNSUPPORTED, "device-counted adaptive evaluations take leaf sizes up to 16384");
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
    need(A.hist, sort_scratch_bytes(n, 63));
    const int64_t tb = (n + kTreeB - 1) / kTreeB;  // one-pass tree blocks
    const int64_t hb = kTreeBins * tb + 1;
    need(A.scan_tmp, 4 * (exclusive_scan_tmp_words(std::max<int64_t>(n + 1, hb)) + 64));
    need(A.flags, 4 * (n + 1));
    need(A.scan, 4 * std::max<int64_t>(n + 1, hb));
    need(A.pcell, 4 * std::max<int64_t>(n, hb));
    need(A.info, 4 * 64);
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
    int32_t *info = A.info.as<int32_t>();
    const int32_t *abort = dev ? info + kInfoAbort : nullptr;
    if (dev) cudaMemsetAsync(info + kInfoAbort, 0, 4, s);

    // ---- box, keys, sort ----
    mark(0);
    const float4 *x = reinterpret_cast<const float4 *>(d_xyzq);
    Box *box = A.box.as<Box>();
    launch_bbox(x, n, prm->has_box, prm->box_origin, prm->box_side, box, partials, counter, ctx->d_status, s);
    k_keys64<<<blocks_for(n), 256, 0, s>>>(x, n, box, A.keys0.as<uint64_t>(), A.idx0.as<uint32_t>());
    note_launches(1);
    mark(1);
    uint64_t *skeys = nullptr;
    uint32_t *perm = nullptr;
    launch_sort_gather64(A.keys0.as<uint64_t>(), A.keys1.as<uint64_t>(), A.idx0.as<uint32_t>(),
                         A.idx1.as<uint32_t>(), n, 63, A.hist.p, ctx->d_status, x, A.sx.as<float4>(), &skeys, &perm,
                         s);
    mark(2);

    // ---- tree ----
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
    std::vector<int> ls;
    int64_t ncells = 0;
    int maxl = 0;
    if (n > 0 && window <= kTreeMaxWindow) {
        // one pass: per-particle level ranges, per-level ranks, one host read of the level sizes
        // (or, under capacities, a device check of them)
        uint16_t *range = A.flags.as<uint16_t>();
        uint32_t *hist = A.scan.as<uint32_t>(), *hbase = reinterpret_cast<uint32_t *>(A.pcell.p);
        k_tree_ranges<<<(unsigned)tb, kTreeB, 2 * (kTreeB + (int)window), s>>>(n, skeys, (int)window, tb, range,
                                                                              hist);
        launch_exclusive_scan(hist, hbase, kTreeBins * tb, A.scan_tmp.as<uint32_t>(), s);
        k_tree_starts<<<1, 32, 0, s>>>(tb, hbase, info);
        note_launches(2);
        if (!dev) {
            int32_t hinfo[kTreeBins + 1];
            cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            ncells = hinfo[kTreeBins - 1];
            A.nleaves = (uint32_t)(hinfo[kTreeBins] - hinfo[kTreeBins - 1]);
            for (int l = 0; l <= kAdaptMaxLevel; ++l)
                if (hinfo[l + 1] > hinfo[l]) maxl = l;
            for (int l = 0; l <= maxl + 1; ++l) ls.push_back(hinfo[l]);
        } else {
            ncells = caps->cells;
            A.nleaves = caps->leaves;
            maxl = caps->maxl;
            GuardCaps g{};
            g.v[0] = caps->cells;
            g.v[1] = caps->leaves;
            for (int l = 0; l <= kAdaptMaxLevel; ++l) g.v[2 + l] = l <= maxl ? caps->level[l] : 0;
            k_guard<<<1, 32, 0, s>>>(info, g, 0, info + kInfoAbort, ctx->d_status);
            note_launches(1);
        }
        if (!cell_bufs(ncells, false, 0) || grow(A.end, 4 * ncells, false, 0, s) ||
            grow(A.leaves, 4 * ncells + 4, false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
        k_tree_cells<<<(unsigned)tb, kTreeB, 0, s>>>(n, skeys, tb, range, hbase, A.level.as<int32_t>(),
                                                     A.key.as<uint64_t>(), A.begin.as<int32_t>(),
                                                     A.parent.as<int32_t>(), A.child_begin.as<int32_t>(),
                                                     A.nchild.as<int32_t>(), A.child_of.as<int32_t>(),
                                                     A.leaves.as<int32_t>(), A.leaf_of.as<int32_t>(), abort);
        const Span cs = dev ? Span{0, ncells, nullptr, info + kTreeBins - 1, abort} : host_span(0, ncells);
        if (ncells > 0)
            k_tree_links<<<blocks_for(ncells), 256, 0, s>>>(cs, n, skeys, info, A.level.as<int32_t>(),
                                                           A.key.as<uint64_t>(), A.begin.as<int32_t>(),
                                                           A.count.as<int32_t>(), A.end.as<int32_t>(),
                                                           A.parent.as<int32_t>(), A.child_begin.as<int32_t>(),
                                                           A.nchild.as<int32_t>(), A.child_of.as<int32_t>());
        k_tree_leaf_of<<<blocks_for(n), 256, 0, s>>>(n, A.leaves.as<int32_t>(), A.leaf_of.as<int32_t>(), abort);
        note_launches(3);
    } else {
        // level by level (leaf sizes beyond the one-pass window, or no particles): one flag /
        // scan / compact round per level, the host reading the number of new cells after each
        if (!cell_bufs(cap, false, 0)) return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
        k_tree_root<<<1, 1, 0, s>>>(n, A.level.as<int32_t>(), A.key.as<uint64_t>(), A.begin.as<int32_t>(),
                                    A.count.as<int32_t>(), A.parent.as<int32_t>(), A.child_begin.as<int32_t>(),
                                    A.nchild.as<int32_t>(), A.child_of.as<int32_t>());
        k_tree_pcell_init<<<blocks_for(n), 256, 0, s>>>(n, A.pcell.as<int32_t>());
        note_launches(2);
        ls = {0, 1};
        ncells = 1;
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
            k_tree_counts<<<blocks_for(nnew), 256, 0, s>>>(ncells, nnew, A.begin.as<int32_t>(),
                                                          A.parent.as<int32_t>(), A.count.as<int32_t>());
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
        if (grow(A.end, 4 * ncells, false, 0, s) || grow(A.leaves, 4 * ncells + 4, false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
        k_cell_end<<<blocks_for(ncells), 256, 0, s>>>(ncells, A.begin.as<int32_t>(), A.count.as<int32_t>(),
                                                     A.end.as<int32_t>());
        note_launches(1);
        cudaMemsetAsync(A.group_cnt.p, 0, A.group_cnt.cap, s);
        uint32_t *leaf_cursor = A.group_cnt.as<uint32_t>() + 8 * (kAdaptMaxLevel + 2) * 2 - 1;
        k_leaf_list<<<blocks_for(ncells), 256, 0, s>>>(ncells, A.nchild.as<int32_t>(), leaf_cursor,
                                                      A.leaves.as<int32_t>());
        note_launches(1);
        A.nleaves = read1<uint32_t>(leaf_cursor, s);
    }
    A.ncells = ncells;
    A.max_level = maxl;
    A.level_start = ls;
    const Ranges R{dev, info, abort, ncells, A.nleaves, &A.level_start, caps};
    if (grow(A.coll, 4 * 27 * ncells, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
    if (grow(A.geom, 16 * (size_t)ncells, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive cells");
    const float4 *geom = A.geom.as<float4>();
    launch_cell_geom(R.cells(), A.level.as<int32_t>(), A.key.as<uint64_t>(), box, A.geom.as<float4>(), s);
    for (int l = 0; l <= maxl; ++l) {
        const Span lv = R.level(l);
        if (lv.cap <= 0) continue;
        k_colleagues<<<blocks_for(lv.cap), 256, 0, s>>>(lv, l, A.key.as<uint64_t>(), A.parent.as<int32_t>(),
                                                       A.child_of.as<int32_t>(), A.coll.as<int32_t>());
        note_launches(1);
    }

    // ---- lists: counts and offsets of the four kinds, one host read of their sizes (or a device
    // check against the capacities), fills ----
    if (grow(A.scan_tmp, 4 * (exclusive_scan_tmp_words(ncells + 1) + 64), false, 0, s))
        return fail(ctx, GBFMM_ENOMEM, "adaptive scan");
    if (grow(A.anchor, 16 * (size_t)ncells, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
    if (ncells > 0) {
        k_cell_anchor<<<blocks_for(ncells), 256, 0, s>>>(R.cells(), A.level.as<int32_t>(), A.key.as<uint64_t>(),
                                                        A.anchor.as<int4>());
        note_launches(1);
    }
    TreeView tv{A.level.as<int32_t>(), A.parent.as<int32_t>(), A.nchild.as<int32_t>(), A.child_of.as<int32_t>(),
                A.coll.as<int32_t>(), A.key.as<uint64_t>(), A.anchor.as<int4>()};
    const unsigned g8 = blocks_for(ncells, 8);
    // U, W, X rows: a warp per cell while the tree is small (latency: the 27 colleague slots in
    // parallel), a thread per cell on large trees (throughput)
    const bool warp_rows = ncells < kListWarpCells;
    const Span cs = R.cells();
    auto launch_alist = [&](int k, bool fill, uint32_t *cnt, const uint32_t *offs, int32_t *ids) {
        const unsigned gt = blocks_for(ncells, 128);
#define GB_ALIST(KIND, FILL)                                                                               \
    (warp_rows ? k_alist_warp<KIND, FILL><<<g8, 256, 0, s>>>(cs, tv, cnt, offs, ids, ctx->d_status)        \
               : k_alist_thread<KIND, FILL><<<gt, 128, 0, s>>>(cs, tv, cnt, offs, ids, ctx->d_status))
        if (k == kListU) {
            if (fill) GB_ALIST(kListU, true); else GB_ALIST(kListU, false);
        } else if (k == kListW) {
            if (fill) GB_ALIST(kListW, true); else GB_ALIST(kListW, false);
        } else {
            if (fill) GB_ALIST(kListX, true); else GB_ALIST(kListX, false);
        }
#undef GB_ALIST
        note_launches(1);
    };
    for (int k = 0; k < 4; ++k) {
        if (grow(A.lcnt[k], 4 * (ncells + 1), false, 0, s) || grow(A.loffs[k], 4 * (ncells + 1), false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
        uint32_t *cnt = A.lcnt[k].as<uint32_t>();
        if (dev) cudaMemsetAsync(cnt, 0, 4 * (ncells + 1), s);  // rows past the cells stay empty
        if (ncells > 0) {
            if (k == kListV)
                k_vlist_warp<false><<<g8, 256, 0, s>>>(cs, tv, cnt, nullptr, nullptr, nullptr);
            else
                launch_alist(k, false, cnt, nullptr, nullptr);
        }
        launch_exclusive_scan(A.lcnt[k].as<uint32_t>(), A.loffs[k].as<uint32_t>(), ncells,
                              A.scan_tmp.as<uint32_t>(), s);
    }
    k_list_totals<<<1, 32, 0, s>>>(ncells, A.loffs[0].as<uint32_t>(), A.loffs[1].as<uint32_t>(),
                                   A.loffs[2].as<uint32_t>(), A.loffs[3].as<uint32_t>(), info + kInfoLists);
    note_launches(1);
    if (!dev) {
        int32_t ltot[4];
        cudaMemcpyAsync(ltot, info + kInfoLists, sizeof(ltot), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        for (int k = 0; k < 4; ++k) A.entries[k] = (uint32_t)ltot[k];
    } else {
        GuardCaps g{};
        for (int k = 0; k < 4; ++k) g.v[k] = A.entries[k] = caps->list[k];
        k_guard<<<1, 32, 0, s>>>(info, g, 1, info + kInfoAbort, ctx->d_status);
        note_launches(1);
    }
    for (int k = 0; k < 4; ++k) {
        const int64_t ne = A.entries[k];
        if (grow(A.lids[k], 4 * (size_t)ne + 4, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
        if (k == kListV && grow(A.vcode, 2 * (size_t)ne + 4, false, 0, s))
            return fail(ctx, GBFMM_ENOMEM, "adaptive lists");
        if (ncells == 0) continue;
        const uint32_t *offs = A.loffs[k].as<uint32_t>();
        int32_t *ids = A.lids[k].as<int32_t>();
        if (k == kListV)
            k_vlist_warp<true><<<g8, 256, 0, s>>>(cs, tv, nullptr, offs, ids, A.vcode.as<uint16_t>());
        else
            launch_alist(k, true, nullptr, offs, ids);
    }
    mark(3);
    A.n = n;
    A.skeys = skeys;
    A.perm = perm;
    if (!dev) {
        AdaptCaps &c = A.counts;
        c = AdaptCaps{};
        c.cells = ncells;
        c.leaves = A.nleaves;
        c.maxl = maxl;
        for (int l = 0; l <= maxl && l + 1 < (int)ls.size(); ++l) c.level[l] = ls[l + 1] - ls[l];
        for (int k = 0; k < 4; ++k) c.list[k] = A.entries[k];
        c.valid = n > 0 && window <= kTreeMaxWindow;
    }
    if (prm->method == GBFMM_METHOD_TREECODE) return treecode_adaptive(ctx, A, R, prm, n, d_out, s, mark);

    // near field beside the far field: P2P (U lists) writes its compensated sums on the
    // context's low-priority stream while the expansions run on its high-priority one (unless
    // the evaluation is timed, serial or device-counted); L2P adds the far field to them and
    // writes the output
    const bool split = p2p_near_supported();
    const bool fork = split && (prm->flags & GBFMM_FLAG_SERIAL) == 0 && !dev;
    ctx->stage_order_last = fork ? 2 : (split ? 1 : 0);
    float4 *near = nullptr;
    if (split) {
        if (grow(A.near, 32 * (size_t)n, false, 0, s)) return fail(ctx, GBFMM_ENOMEM, "adaptive near field");
        near = A.near.as<float4>();
    }
    const cudaStream_t s_main = s;
    // an error after the fork still joins both streams back into the caller's
    auto fail_joined = [&](int code, const char *msg) {
        if (fork) {
            cudaEventRecord(ctx->ev_join, ctx->s_far);
            cudaStreamWaitEvent(s_main, ctx->ev_join, 0);
            cudaStreamWaitEvent(s_main, ctx->ev_near, 0);
        }
        return fail(ctx, code, msg);
    };
    if (fork) {
        cudaEventRecord(ctx->ev_fork, s_main);
        cudaStreamWaitEvent(ctx->s_far, ctx->ev_fork, 0);
        cudaStreamWaitEvent(ctx->s_near, ctx->ev_fork, 0);
        s = ctx->s_far;
        if (timing) cudaEventRecord(ctx->ev_aux[0], ctx->s_near);
        launch_p2p_cells_near(A.leaves.as<int32_t>(), R.leaves(), n, A.sx.as<float4>(), A.begin.as<int32_t>(),
                              A.end.as<int32_t>(), A.loffs[kListU].as<uint32_t>(), A.lids[kListU].as<int32_t>(),
                              (float)prm->eps2, near, ctx->d_status, ctx->s_near);
        if (timing) cudaEventRecord(ctx->ev_aux[1], ctx->s_near);
        cudaEventRecord(ctx->ev_near, ctx->s_near);
    }

    // ---- expansions ----
    if (grow(A.M, 4 * (size_t)ncells * PP, false, 0, s) || grow(A.Lc, 4 * (size_t)ncells * PP, false, 0, s))
        return fail_joined(GBFMM_ENOMEM, "adaptive expansions");
    float *M = A.M.as<float>(), *Lc = A.Lc.as<float>();
    float4 *far = A.far.as<float4>();
    const bool deep = maxl >= 2;
    if (deep) launch_p2m_cells(P, A.leaves.as<int32_t>(), R.leaves(), A.level.as<int32_t>(), geom,
                               A.begin.as<int32_t>(), A.count.as<int32_t>(), A.sx.as<float4>(), M, s);
    mark(4);
    for (int l = maxl - 1; l >= 2; --l)
        launch_translate_cells(P, true, R.level(l), A.child_of.as<int32_t>(), A.nchild.as<int32_t>(), ops.m2m, M, s);
    mark(5);
    const bool cores = (prm->flags & GBFMM_FLAG_M2L_CUDA_CORES) != 0;
    const bool gathered = (prm->flags & GBFMM_FLAG_M2L_GATHERED) != 0;
    if (deep && !cores && !gathered) {
        // M2L in block form: one GEMM per parent offset over the units (cells with children),
        // their colleagues' children gathered per tile; no V list is read
        rc = ensure_blk(ctx, P, s);
        if (rc != GBFMM_OK) return fail_joined(rc, "block operators");
        const int64_t ucap = dev ? ncells : std::max<int64_t>(1, ncells - A.nleaves);
        const int64_t up = m2l_ablk_tiles_units(ucap);
        if (grow(A.ab_flag, 4 * (size_t)(ncells + 1), false, 0, s) || grow(A.ab_scan, 4 * (size_t)(ncells + 1), false, 0, s) ||
            grow(A.ab_unit_of, 4 * (size_t)ncells + 4, false, 0, s) || grow(A.ab_units, 4 * (size_t)up + 4, false, 0, s) ||
            grow(A.ab_nu, 16, false, 0, s) || grow(A.ab_pre, m2l_ablk_presplit_bytes(P, ucap), false, 0, s) ||
            grow(A.ab_scale, (size_t)ucap + 16, false, 0, s) || grow(A.ab_src, m2l_ablk_src_bytes(ucap), false, 0, s))
            return fail_joined(GBFMM_ENOMEM, "block M2L buffers");
        const int ksplit = m2l_ablk_ksplit(P, n, prm->leaf_size);
        const int64_t part_stride = ncells * PP;
        if (ksplit > 1 && grow(A.lpart, 4 * (size_t)ksplit * part_stride, false, 0, s))
            return fail_joined(GBFMM_ENOMEM, "block M2L partial sums");
        launch_ablk_prep(P, R.cells(), ucap, A.level.as<int32_t>(), A.nchild.as<int32_t>(), A.child_of.as<int32_t>(),
                         A.coll.as<int32_t>(), M, A.ab_flag.as<uint32_t>(), A.ab_scan.as<uint32_t>(),
                         A.scan_tmp.as<uint32_t>(), A.ab_unit_of.as<int32_t>(), A.ab_units.as<int32_t>(),
                         A.ab_nu.as<int32_t>(), A.ab_pre.p, A.ab_scale.as<int8_t>(), A.ab_src.as<int32_t>(), s);
        if (launch_m2l_ablk(P, ucap, A.ab_nu.as<int32_t>(), A.ab_units.as<int32_t>(), A.child_of.as<int32_t>(),
                            A.ab_src.as<int32_t>(), A.ab_pre.p, A.ab_scale.as<int8_t>(), ops.m2l_blk, Lc,
                            ksplit > 1 ? A.lpart.as<float>() : nullptr, ksplit, part_stride, ctx->d_status, s,
                            fork ? sm_count() : 0) != 0)
            return fail_joined(GBFMM_ECUDA, "TMA tensor map encoding failed");
        if (ksplit > 1) launch_ablk_reduce(P, R.deep(), ksplit, part_stride, A.lpart.as<float>(), Lc, s);
        launch_p2l_cells(P, R.cells(), A.level.as<int32_t>(), geom, A.begin.as<int32_t>(), A.count.as<int32_t>(),
                         A.loffs[kListX].as<uint32_t>(), A.lids[kListX].as<int32_t>(), A.sx.as<float4>(), Lc, s);
    } else if (deep) {
        // M2L targets: every cell at levels >= 2, grouped by (level, child position) into tiles
        // planned on the device (no host read); launched over a bound on the tile count, tiles
        // past the last one empty
        const Span dp = R.deep();
        uint32_t *gcnt = A.group_cnt.as<uint32_t>();
        uint32_t *gcur = gcnt + 8 * (kAdaptMaxLevel + 2);
        cudaMemsetAsync(gcnt, 0, 4 * 8 * (kAdaptMaxLevel + 2), s);
        if (dp.cap > 0) {
            k_group_count<<<blocks_for(dp.cap), 256, 0, s>>>(dp, A.level.as<int32_t>(), A.key.as<uint64_t>(), gcnt);
            note_launches(1);
        }
        const bool f16 = !cores;
        const int TN = f16 ? kM2LTcTargetsPerTile : kM2LTargetsPerTile;
        const int64_t tcap = dp.cap / TN + 8 * (int64_t)(maxl - 1) + 1;
        if (grow(A.tlist, 4 * (size_t)dp.cap + 4, false, 0, s) || grow(A.tdesc, sizeof(int4) * tcap + 16, false, 0, s))
            return fail_joined(GBFMM_ENOMEM, "adaptive tiles");
        k_tile_plan<<<1, 256, 0, s>>>(gcnt, gcur, A.tdesc.as<int4>(), tcap, TN, abort);
        note_launches(1);
        if (dp.cap > 0) {
            k_group_fill<<<blocks_for(dp.cap), 256, 0, s>>>(dp, A.level.as<int32_t>(), A.key.as<uint64_t>(), gcur,
                                                           A.tlist.as<int32_t>());
            note_launches(1);
        }
        if (f16) {
            if (grow(A.cscale, (size_t)ncells + 16, false, 0, s)) return fail_joined(GBFMM_ENOMEM, "adaptive scales");
            if (grow(A.presplit, presplit_bytes(P, ncells), false, 0, s))
                return fail_joined(GBFMM_ENOMEM, "adaptive pre-split sources");
            void *ps = A.presplit.p;
            launch_presplit(P, M, ncells, A.cscale.as<int8_t>(), ps, s, R.cells());  // sources split once per cell
            launch_m2l_f16_tiles(P, A.tdesc.as<int4>(), (int)tcap, A.tlist.as<int32_t>(), A.begin.as<int32_t>(),
                                 A.end.as<int32_t>(), A.loffs[kListV].as<uint32_t>(), A.lids[kListV].as<int32_t>(),
                                 A.vcode.as<uint16_t>(), ops.m2l_f16, M, A.cscale.as<int8_t>(), ps, Lc,
                                 ctx->d_status, s, fork ? sm_count() : 0);
        } else
            launch_m2l_tiles(P, A.tdesc.as<int4>(), (int)tcap, A.tlist.as<int32_t>(), A.begin.as<int32_t>(),
                             A.end.as<int32_t>(), A.loffs[kListV].as<uint32_t>(), A.lids[kListV].as<int32_t>(),
                             A.vcode.as<uint16_t>(), ops.m2l, M, Lc, ctx->d_zero, ctx->d_status, s);
        launch_p2l_cells(P, R.cells(), A.level.as<int32_t>(), geom, A.begin.as<int32_t>(), A.count.as<int32_t>(),
                         A.loffs[kListX].as<uint32_t>(), A.lids[kListX].as<int32_t>(), A.sx.as<float4>(), Lc, s);
    }
    mark(6);
    for (int l = 3; l <= maxl; ++l)
        launch_translate_cells(P, false, R.level(l - 1), A.child_of.as<int32_t>(), A.nchild.as<int32_t>(), ops.l2l,
                               Lc, s);
    mark(7);
    if (split) {
        // M2P into the zeroed far field, then L2P adds the local expansion's value and the
        // near-field sums (the same rounding as L2P then M2P: one addition each)
        if (!fork) {
            launch_p2p_cells_near(A.leaves.as<int32_t>(), R.leaves(), n, A.sx.as<float4>(), A.begin.as<int32_t>(),
                                  A.end.as<int32_t>(), A.loffs[kListU].as<uint32_t>(), A.lids[kListU].as<int32_t>(),
                                  (float)prm->eps2, near, ctx->d_status, s);
            mark(8);
        }
        cudaMemsetAsync(far, 0, 16 * (size_t)n, s);
        if (deep)
            launch_m2p_cells(P, A.leaves.as<int32_t>(), R.leaves(), geom, A.begin.as<int32_t>(),
                             A.end.as<int32_t>(), A.loffs[kListW].as<uint32_t>(), A.lids[kListW].as<int32_t>(),
                             A.sx.as<float4>(), M, far, s);
        if (fork) {
            mark(8);
            cudaStreamWaitEvent(s, ctx->ev_near, 0);
            if (timing) cudaEventRecord(ctx->ev_aux[2], s);
        }
        launch_l2p_cells(P, n, A.leaf_of.as<int32_t>(), A.level.as<int32_t>(), geom, A.sx.as<float4>(), Lc, far, s,
                         near, perm, reinterpret_cast<float4 *>(d_out), abort);
        mark(9);
        if (fork) {
            cudaEventRecord(ctx->ev_join, s);
            cudaStreamWaitEvent(s_main, ctx->ev_join, 0);
            s = s_main;
        }
    } else {
        launch_l2p_cells(P, n, A.leaf_of.as<int32_t>(), A.level.as<int32_t>(), geom, A.sx.as<float4>(), Lc, far, s,
                         nullptr, nullptr, nullptr, abort);
        if (deep)
            launch_m2p_cells(P, A.leaves.as<int32_t>(), R.leaves(), geom, A.begin.as<int32_t>(),
                             A.end.as<int32_t>(), A.loffs[kListW].as<uint32_t>(), A.lids[kListW].as<int32_t>(),
                             A.sx.as<float4>(), M, far, s);
        mark(8);
        launch_p2p_cells(A.leaves.as<int32_t>(), R.leaves(), n, A.sx.as<float4>(), A.begin.as<int32_t>(),
                         A.end.as<int32_t>(), A.loffs[kListU].as<uint32_t>(), A.lids[kListU].as<int32_t>(), far, perm,
                         (float)prm->eps2, reinterpret_cast<float4 *>(d_out), ctx->d_status, s);
        mark(9);
    }
    A.P = P;
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
    // the treecode forms no local expansions: those export as zeros
    const bool any = A.max_level >= 2 && (which == 0 || ctx->last_method == GBFMM_METHOD_FMM);
    if (any) cudaMemcpy(v.data(), which == 0 ? A.M.p : A.Lc.p, 4 * v.size(), cudaMemcpyDeviceToHost);
    cudaMemcpy(lev.data(), A.level.p, 4 * nc, cudaMemcpyDeviceToHost);
    for (size_t c = 0; c < nc; ++c) {
        const int l = lev[c];
        const double h = box.side / (double)(int64_t(1) << l);
        const bool formed = any && l >= 2;
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
