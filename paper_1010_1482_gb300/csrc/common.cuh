// Internal declarations shared by the CUDA translation units of libgbfmm.
//
// Data layout in device memory (one evaluation, uniform octree of depth L):
//   cells: dense per level, the level-l cell with Morton key k at global index
//          level_offset(l) + k, level_offset(l) = (8^l - 1) / 7;
//   expansions: real-packed, P*P floats per cell: degree n occupies
//          [n*n, (n+1)*(n+1)) as Re C_n^0, Re C_n^1, Im C_n^1, ..., Re C_n^n, Im C_n^n
//          (C_n^{-m} = conj(C_n^m) is implied, Im C_n^0 = 0 is dropped);
//          stored scaled by the cell side h of their level: M~_n^m = M_n^m / h^n,
//          L~_n^m = L_n^m h^(n+1), so every translation operator is independent of
//          the level and is tabulated once per order p.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GB_DEV __device__ __forceinline__
#define GB_HD __host__ __device__ __forceinline__

namespace gbfmm {

constexpr int kMaxLevel = 10;
constexpr int kM2LCodes = 343;  // offsets (dx, dy, dz) in [-3, 3]^3, code = (dx+3) + 7(dy+3) + 49(dz+3)

GB_HD int64_t level_offset(int l) { return ((int64_t(1) << (3 * l)) - 1) / 7; }

GB_HD int m2l_code(int dx, int dy, int dz) { return (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3); }

// Morton interleave of three 10-bit integers (bit 3b+0 = x bit b, 3b+1 = y, 3b+2 = z).
GB_HD uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

GB_HD uint32_t compact3(uint32_t v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}

GB_HD uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) { return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2); }

GB_HD void demorton3(uint32_t k, int &x, int &y, int &z)
{
    x = (int)compact3(k);
    y = (int)compact3(k >> 1);
    z = (int)compact3(k >> 2);
}

// 63-bit Morton interleave of three 21-bit integers (same bit order as morton3).
GB_HD uint64_t spread21(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

GB_HD uint64_t compact21(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return v;
}

GB_HD uint64_t morton63(uint64_t x, uint64_t y, uint64_t z) { return spread21(x) | (spread21(y) << 1) | (spread21(z) << 2); }

// integer coordinates of the level-l cell whose key prefix is `key` (3l bits)
GB_HD void demorton63(uint64_t key, int &x, int &y, int &z)
{
    x = (int)compact21(key);
    y = (int)compact21(key >> 1);
    z = (int)compact21(key >> 2);
}

// Translation-operator tables (M2L, M2M, L2L) are stored column-major, [op][col][row], with
// the row count padded to a multiple of 8 (zero rows), so row blocks of 4 or 8 per thread
// stay 16-byte aligned.
GB_HD constexpr int ops_rows_padded(int P) { return (P * P + 7) / 8 * 8; }

// stride (floats) of a staged expansion column in shared memory: a multiple of 4 with
// (stride / 4) odd, so the 16-byte column reads of eight consecutive columns fall in distinct
// bank groups
GB_HD constexpr int staged_col_stride(int P) { return ((P * P / 4) % 2 == 1) ? P * P : P * P + 4; }

// Register fragments of one k-group (4 consecutive k): CN staged source columns (4 k each)
// and RM operator rows for each of the 4 k.
template <int CN, int RM>
struct Frag {
    float4 b[CN];
    float4 a[4][RM / 4];
    GB_DEV void load(const float *A, const float *B, int k, int PR, int bstride)
    {
#pragma unroll
        for (int j = 0; j < CN; ++j) b[j] = *reinterpret_cast<const float4 *>(B + j * bstride + k);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int qq = 0; qq < RM / 4; ++qq) a[kk][qq] = *reinterpret_cast<const float4 *>(A + (k + kk) * PR + 4 * qq);
    }
    // k outer, targets and rows inner: consecutive FMAs update different accumulators
    // (RM x CN independent chains per k)
    __device__ __forceinline__ void fma(float (&acc)[RM][CN]) const
    {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int j = 0; j < CN; ++j) {
                const float bv = kk == 0 ? b[j].x : kk == 1 ? b[j].y : kk == 2 ? b[j].z : b[j].w;
#pragma unroll
                for (int qq = 0; qq < RM / 4; ++qq) {
                    acc[4 * qq + 0][j] = fmaf(a[kk][qq].x, bv, acc[4 * qq + 0][j]);
                    acc[4 * qq + 1][j] = fmaf(a[kk][qq].y, bv, acc[4 * qq + 1][j]);
                    acc[4 * qq + 2][j] = fmaf(a[kk][qq].z, bv, acc[4 * qq + 2][j]);
                    acc[4 * qq + 3][j] = fmaf(a[kk][qq].w, bv, acc[4 * qq + 3][j]);
                }
            }
    }
};

// Device status bits (OR-ed into the context's status word).
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusCapacity = 4;  // a captured adaptive evaluation outgrew its capacities

// The items one launch covers.  The grid spans `cap` items; the kernel takes count() of them,
// starting at first().  With no device pointers this is [lo, lo + cap) as launched (counts the
// host knows); with them, the range [*dlo, *dhi) is read on the device and clamped to cap, and
// it is empty once *abort is nonzero (counts only the device knows: captured evaluations).
struct Span {
    int64_t lo = 0, cap = 0;
    const int32_t *dlo = nullptr, *dhi = nullptr, *abort = nullptr;
};
inline Span host_span(int64_t lo, int64_t n) { return Span{lo, n < 0 ? 0 : n, nullptr, nullptr, nullptr}; }
GB_DEV int64_t span_first(const Span &s) { return s.dlo ? (int64_t)*s.dlo : s.lo; }
GB_DEV int64_t span_count(const Span &s)
{
    if (s.abort && *s.abort) return 0;
    if (!s.dhi) return s.cap;
    const int64_t n = (int64_t)*s.dhi - span_first(s);
    return n < 0 ? 0 : (n < s.cap ? n : s.cap);
}

// compensated (Kahan) summation: s the running sum, c the lost low-order part
struct Kahan {
    float s, c;
    GB_DEV void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// The hardware reciprocal square root (rsqrt.approx.ftz: relative error about 2^-23, subnormal
// inputs flushed).  The pair rules and the far-field series take it on squared distances that
// are either zero (masked by the caller) or far above the subnormal range.
GB_DEV float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Root box as computed on the device: origin xyz and side, FP64.
struct Box {
    double origin[3];
    double side;
    double key_scale;  // 2^21 / side, one IEEE FP64 division
    // FP32 roundings of origin and key_scale, and the slack of the FP32 key estimate (k_keys):
    // |FP32 estimate - FP64 value| <= |estimate| 2^-21 + key_slack
    float origin_f[3];
    float key_scale_f;
    float key_slack;
    // the FP32 roundings of origin - origin_f and key_scale - key_scale_f: with them the origin and
    // the scale as float-float pairs (the 63-bit keys' estimate, grid_coord21)
    float origin_lo[3];
    float key_scale_lo;
};

// k = clamp(floor((c - origin) * scale), 0, 2^21 - 1) with every step one IEEE FP64 rounding
// (NaN maps to 0): the key coordinate at depth 21.  Not inlined: the key kernels call it for the
// rare coordinates their FP32 estimates cannot decide, and a real branch keeps the FP64
// instructions (slow on this part) off the path of every other lane.
static __device__ __noinline__ uint32_t grid_coord_fp64(float c, double origin, double scale)
{
    double t = __dsub_rn((double)c, origin);
    double v = __dmul_rn(t, scale);
    double f = floor(v);
    if (!(f >= 0.0)) f = 0.0;  // also maps NaN to 0
    if (f > 2097151.0) f = 2097151.0;
    return (uint32_t)f;
}

// The same coordinate from a float-float estimate of the real w = (c - o) s (o = origin_f +
// origin_lo, s = key_scale_f + key_scale_lo): p + e with p = RN(th sh), e its product error plus
// the low parts, th + tl = c - origin_f exactly (two-sum).  The estimate is within 2^-45 (|o| s +
// |w|) of w and the FP64 value within 2^-52 |w| of w; with f = floor(RN(p + e)), moved by one
// when that rounding crossed an integer, and r = (p - f) + e (p - f exact, at most two roundings
// of 2^-24 after it), both floors are f when r lies at least E = 2^-44 (|o| s + |p|) + 2^-22
// inside (0, 1).  Otherwise, and for |p| >= 2^22 or a non-finite
// coordinate, the FP64 steps decide.
GB_DEV uint32_t grid_coord21(float c, const Box &b, int d)
{
    const float oh = b.origin_f[d], ol = b.origin_lo[d], sh = b.key_scale_f, sl = b.key_scale_lo;
    const float th = __fsub_rn(c, oh);
    const float bv = __fsub_rn(th, c);
    const float tl = __fadd_rn(__fsub_rn(c, __fsub_rn(th, bv)), __fsub_rn(-oh, bv));
    const float tl2 = __fsub_rn(tl, ol);
    const float p = __fmul_rn(th, sh);
    const float e1 = __fmaf_rn(th, sh, -p);
    const float e2 = __fadd_rn(__fmul_rn(th, sl), __fmul_rn(tl2, sh));
    const float e = __fadd_rn(e1, e2);
    if (fabsf(p) < 4194304.f) {
        // RN(p + e) can round across an integer (its unit in the last place is up to 1/4):
        // one step back or forward puts r in [0, 1)
        float f = floorf(__fadd_rn(p, e));
        float r = __fadd_rn(__fsub_rn(p, f), e);
        if (r < 0.f) {
            f = __fsub_rn(f, 1.f);
            r = __fadd_rn(r, 1.f);
        } else if (r >= 1.f) {
            f = __fadd_rn(f, 1.f);
            r = __fsub_rn(r, 1.f);
        }
        const float E = __fadd_ru(__fmul_ru(__fadd_ru(__fmul_ru(fabsf(oh), sh), fabsf(p)), 0x1p-44f), 0x1p-22f);
        if (r >= E && r <= __fsub_rd(1.f, E)) return f < 0.f ? 0u : (f > 2097151.f ? 2097151u : (uint32_t)f);
    }
    return grid_coord_fp64(c, b.origin[d], b.key_scale);
}

// Cell geometry table of the uniform tree (expansions.cu, k_geo_levels): 1/h_l for
// l < kGeoLevels, then the 2^l cell-centre coordinates of every level l = 0..L along x, y, z.
constexpr int kGeoLevels = 22;
inline size_t geo_floats(int L) { return kGeoLevels + 3 * ((size_t(2) << L) - 1); }

// Layout of one evaluation's workspace (byte offsets from the workspace base).
struct Layout {
    int64_t n;
    int L;
    int P;
    int64_t ncells;     // C
    int64_t nleaves;    // 8^L
    int64_t rs_blocks;  // radix-sort tiles
    size_t box, status_dummy;
    size_t keys0, keys1, idx0, idx1;
    size_t sx, far;
    size_t rs_hist, scan_tmp;
    size_t cell_begin, cell_end;
    size_t p2p_len, p2p_offs, p2p_ids;
    size_t m2l_len, m2l_offs, m2l_ids, m2l_code;
    size_t M, Lc;
    size_t cscale;  // int8 per cell: power-of-two scale of the FP16 tensor-core M2L
    size_t geo;       // float: cell geometry table per level and axis (geo_floats(L))
    size_t presplit;  // FP16 pre-split source rows of the tensor-core M2L (gathered or block form)
    size_t lpart;     // block M2L of small trees: partial local expansions of the offset ranges
    size_t total;
};

// Kernel-launch accounting: every launcher reports the kernels it enqueued (api.cu keeps the
// count of the current evaluation).
void note_launches(int k);

// ---- launchers (host functions, one per device stage) -------------------------------------
// tree.cu
void launch_bbox(const float4 *x, int64_t n, int has_box, const double *box_origin, double box_side, Box *box_out,
                 float *partials, unsigned *counter, int *status, cudaStream_t s);
void launch_keys(const float4 *x, int64_t n, const Box *box, int L, uint32_t *leafkey, uint32_t *idx, cudaStream_t s);
// Radix-sort scratch (tree.cu): per-pass tile counters, the histograms of every 8-bit digit
// position, and one 64-bit look-back word per (pass, tile of 4096 keys, digit).
constexpr size_t kRsCounterBytes = 256, kRsHistBytes = 8 * 256 * 4;
constexpr size_t sort_scratch_bytes(int64_t n, int bits)
{
    return kRsCounterBytes + kRsHistBytes + 8 * 256 * (size_t)((bits + 7) / 8) * (size_t)((n + 4095) / 4096);
}
// sorts (keys, idx) by key (stable) over `bits` low bits (keys < 2^bits); on return the sorted
// pair is in (*keys_out, *idx_out) (one of the two buffers); also gathers sx[i] = x[idx[i]].
// `scratch` holds sort_scratch_bytes(n, bits); a look-back wait that runs out raises
// kStatusTimeout in *err.
void launch_sort_gather(uint32_t *k0, uint32_t *k1, uint32_t *v0, uint32_t *v1, int64_t n, int bits, void *scratch,
                        int *err, const float4 *x, float4 *sx, uint32_t **keys_out, uint32_t **idx_out,
                        cudaStream_t s);
void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s);
size_t exclusive_scan_tmp_words(int64_t n);
void launch_cells(const uint32_t *sorted_leaf_keys, int64_t n, int L, int32_t *begin, int32_t *end, cudaStream_t s);
void launch_list_count(int L, const int32_t *begin, const int32_t *end, uint32_t *p2p_len, uint32_t *m2l_len,
                       cudaStream_t s);
void launch_list_fill(int L, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs, int32_t *p2p_ids,
                      const uint32_t *m2l_offs, int32_t *m2l_ids, uint16_t *m2l_code, cudaStream_t s);
// the P2P rows alone (the block M2L of the uniform tree reads no M2L list)
void launch_p2p_list_count(int L, const int32_t *begin, const int32_t *end, uint32_t *p2p_len, cudaStream_t s);
void launch_p2p_list_fill(int L, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs, int32_t *p2p_ids,
                          cudaStream_t s);

// expansions.cu
void launch_build_operators(int P, float *m2l_ops, float *m2m_ops, float *l2l_ops, cudaStream_t s);
void launch_geo_levels(const Box *box, int L, float *geo, cudaStream_t s);
void launch_p2m(int P, int L, const float *geo, const float4 *sx, const int32_t *begin, const int32_t *end, float *M,
                cudaStream_t s);
void launch_m2m(int P, int l, const int32_t *begin, const int32_t *end, const float *ops, float *M, cudaStream_t s);
void launch_l2l(int P, int l, const int32_t *begin, const int32_t *end, const float *ops, float *Lc, cudaStream_t s);
// near != nullptr: add the P2P kernel's compensated near-field sums (launch_p2p_near) and write
// the total to out[perm[i]] instead of far[i]
void launch_l2p(int P, int L, const float *geo, int64_t n, const float4 *sx, const uint32_t *leafkey, const float *Lc,
                float4 *far, cudaStream_t s, const float4 *near = nullptr, const uint32_t *perm = nullptr,
                float4 *out = nullptr);
void launch_m2p(int P, int L, const float *geo, const float4 *sx, const int32_t *begin, const int32_t *end,
                const uint32_t *m2l_offs, const int32_t *m2l_ids, const float *M, float4 *far, cudaStream_t s);

// m2l.cu
constexpr int kM2LTargetsPerTile = 64;  // targets per M2L CTA (tile list mode)
void launch_m2l(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                const int32_t *m2l_ids, const uint16_t *m2l_code, const float *ops, const float *M, float *Lc,
                const float *zero_block, int *status, cudaStream_t s);

void launch_wait_selftest(uint64_t limit_ns, int *status, cudaStream_t s);

// adaptive tree (targets and sources given as cell lists; cells carry level and 63-bit key)
void launch_sort_gather64(uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, int64_t n, int bits,
                          void *scratch, int *err, const float4 *x, float4 *sx, uint64_t **keys_out,
                          uint32_t **idx_out, cudaStream_t s);
// Cell launches over the adaptive tree take their cells as a Span (cells c = first() + i), leaf
// launches their leaves as a Span over the leaf list (leaf ordinals i < count()).
void launch_cell_geom(Span cells, const int32_t *level, const uint64_t *key, const Box *box, float4 *geom,
                      cudaStream_t s);
void launch_p2m_cells(int P, const int32_t *leaves, Span lv, const int32_t *level, const float4 *geom,
                      const int32_t *begin, const int32_t *count, const float4 *sx, float *M, cudaStream_t s);
// parents: the cells whose children are translated (M2M up into them, L2L down from them)
void launch_translate_cells(int P, bool up, Span parents, const int32_t *child_of, const int32_t *nchild,
                            const float *ops, float *X, cudaStream_t s);
// tile lists (tdesc: level, child position, first target in tlist, target count): tiles with a
// count of 0 are empty and return at once
void launch_m2l_tiles(int P, const int4 *tdesc, int ntiles, const int32_t *tlist, const int32_t *begin,
                      const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids, const uint16_t *m2l_code,
                      const float *ops, const float *M, float *Lc, const float *zero_block, int *status,
                      cudaStream_t s);
// M2L on the tcgen05 tensor cores (3xTF32 or 3xF16), 128 targets per CTA
constexpr int kM2LTcTargetsPerTile = 128;
size_t m2l_f16_table_bytes(int P);
void launch_build_m2l_f16(int P, const float *ops, void *table, cudaStream_t s);
// max_ctas > 0: the tiles are launched max_ctas at a time (one wave of one CTA per SM), so that
// no CTA of the M2L waits for an SM while a kernel on another stream (the near field) could use
// the room left beside the running ones
void launch_m2l_f16(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                    const int32_t *m2l_ids, const uint16_t *m2l_code, const void *table, const float *M,
                    const int8_t *cscale, const void *ps, float *Lc, int *status, cudaStream_t s, int max_ctas = 0);
void launch_m2l_f16_tiles(int P, const int4 *tdesc, int ntiles, const int32_t *tlist, const int32_t *begin,
                          const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                          const uint16_t *m2l_code, const void *table, const float *M, const int8_t *cscale,
                          const void *ps, float *Lc, int *status, cudaStream_t s, int max_ctas = 0);
// number of SMs of the current device (cached per process)
int sm_count();
// per cell: the FP16 scale s_c and the pre-split halves of M~_c 2^s_c (KP / 8 pieces of 8 hi
// then 8 lo halves), the sources of the list-based FP16 M2L
size_t presplit_bytes(int P, int64_t ncells);
void launch_presplit(int P, const float *M, int64_t ncells, int8_t *scale, void *ps, cudaStream_t s,
                     Span cells = Span{});
void launch_p2l_cells(int P, Span cells, const int32_t *level, const float4 *geom, const int32_t *begin,
                      const int32_t *count, const uint32_t *x_offs, const int32_t *x_ids, const float4 *sx, float *Lc,
                      cudaStream_t s);
// near != nullptr: far holds the M2P sums; the local expansion's value, those and the near-field
// sums are added and written to out[perm[i]].  Nothing runs once *abort is nonzero.
void launch_l2p_cells(int P, int64_t n, const int32_t *leaf_of, const int32_t *level, const float4 *geom,
                      const float4 *sx, const float *Lc, float4 *far, cudaStream_t s, const float4 *near = nullptr,
                      const uint32_t *perm = nullptr, float4 *out = nullptr, const int32_t *abort = nullptr);
// long_rows: the treecode's chain rows (the warp kernel, k_m2p_warp); else the FMM's short W
// rows (one CTA of 64 per leaf, k_m2p_cells)
void launch_m2p_cells(int P, const int32_t *leaves, Span lv, const float4 *geom, const int32_t *begin,
                      const int32_t *end, const uint32_t *w_offs, const int32_t *w_ids, const float4 *sx,
                      const float *M, float4 *far, cudaStream_t s, bool long_rows = false);
void launch_p2p_cells(const int32_t *leaves, Span lv, int64_t n, const float4 *sx, const int32_t *begin,
                      const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, const float4 *far,
                      const uint32_t *perm, float eps2, float4 *out, int *status, cudaStream_t s);

// m2l_blk.cu: the uniform tree's M2L as one dense GEMM per parent offset on the tensor cores
size_t m2l_blk_table_bytes(int P);
void launch_build_m2l_blk(int P, const float *ops, void *table, cudaStream_t s);
size_t m2l_blk_presplit_bytes(int P, int L);
size_t m2l_blk_scale_bytes(int L);
void launch_blk_presplit(int P, int L, const int32_t *begin, const int32_t *end, const float *M, void *presplit,
                         int8_t *pscale, cudaStream_t s);
// small trees split the 26 parent offsets over several CTAs per tile; their partial sums take
// m2l_blk_part_bytes of workspace and are added in a fixed order
int m2l_blk_ksplit(int P, int L);
size_t m2l_blk_part_bytes(int P, int L);
// -1 if the TMA tensor maps cannot be encoded (nothing launched)
int launch_m2l_blk(int P, int L, const int32_t *begin, const int32_t *end, const void *presplit, const int8_t *pscale,
                   const void *table, float *Lc, float *Lpart, int *status, cudaStream_t s, int max_ctas);

// m2l_blk.cu, adaptive tree: the block form over units (cells of levels >= 1 with children;
// ucap >= their count, zrow = ucap the zero row)
size_t m2l_ablk_presplit_bytes(int P, int64_t ucap);
size_t m2l_ablk_src_bytes(int64_t ucap);
int64_t m2l_ablk_tiles_units(int64_t ucap);
int m2l_ablk_ksplit(int P, int64_t n, int leaf_size);
void launch_ablk_prep(int P, Span cells, int64_t ucap, const int32_t *level, const int32_t *nchild,
                      const int32_t *child_of, const int32_t *coll, const float *M, uint32_t *flag, uint32_t *scan,
                      uint32_t *scan_tmp, int32_t *unit_of, int32_t *units, int32_t *n_units, void *Apre,
                      int8_t *uscale, int32_t *src, cudaStream_t s);
// -1 if the operators' tensor map cannot be encoded (nothing launched)
int launch_m2l_ablk(int P, int64_t ucap, const int32_t *n_units, const int32_t *units, const int32_t *child_of,
                    const int32_t *src, const void *Apre, const int8_t *uscale, const void *table, float *Lc,
                    float *Lpart, int ksplit, int64_t part_stride, int *status, cudaStream_t s, int max_ctas);
void launch_ablk_reduce(int P, Span deep, int ksplit, int64_t part_stride, const float *Lpart, float *Lc,
                        cudaStream_t s);

// m2l_rot.cu: the M2L by rotation to the translation axis (O(p^3) per pair, FP32 CUDA cores)
void init_m2l_rot_constants();
size_t m2l_rot_table_bytes(int P);
int build_m2l_rot(int P, void *table);  // host FP64 factors, checked, copied to the device; 0 = OK
void launch_m2l_rot(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                    const int32_t *m2l_ids, const uint16_t *m2l_code, const void *table, const float *M, float *Lc,
                    cudaStream_t s);

// p2p.cu
// P2P without the far field: the compensated near-field sums of every particle in sorted order,
// near[2 i] = sums (phi, dphi/dx, dphi/dy, dphi/dz), near[2 i + 1] = their compensations (the
// warp-specialised kernel: p2p_near_supported()).  The P2P launchers take the context's status
// word: a bounded wait that expires raises kStatusTimeout there.
bool p2p_near_supported();
// P2P launch shape for the launches this thread issues next: about `leaves` target leaves per
// CTA (0: the library's choice; at most kMaxP2PLeavesPerCta); the results do not depend on it
constexpr int kMaxP2PLeavesPerCta = 64;
void set_p2p_leaves_per_cta(int leaves);
void launch_p2p_near(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end,
                     const uint32_t *p2p_offs, const int32_t *p2p_ids, float eps2, float4 *near, int *status,
                     cudaStream_t s);
void launch_p2p_cells_near(const int32_t *leaves, Span lv, int64_t n, const float4 *sx, const int32_t *begin,
                           const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, float eps2, float4 *near,
                           int *status, cudaStream_t s);
void launch_p2p(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end,
                const uint32_t *p2p_offs, const int32_t *p2p_ids, const float4 *far, const uint32_t *perm, float eps2,
                float4 *out, int *status, cudaStream_t s);
void launch_direct(int64_t n_src, const float4 *src, int64_t n_tgt, const float4 *tgt, float eps2, float4 *out,
                   cudaStream_t s);

}  // namespace gbfmm
