// Tree front end of the FMM on the device: root box, Morton keys, stable radix sort of the
// particles by leaf key, per-level cell ranges and the CSR interaction lists.
//
// The paper runs these steps ("sort" and "other": tree construction and list generation) on
// the host (Section "Improvements of Performance", Fig. 5); here every one is an integer or
// bandwidth-bound device kernel.  This translation unit is compiled with -fmad=false and the
// key quantisation uses explicit IEEE round-to-nearest FP64 intrinsics, so the keys are the
// exact result of floor((x - origin) * (2^21 / side)) and match any IEEE FP64 evaluation of
// the same steps bit for bit.
#include "common.cuh"

#include <math.h>

#include <algorithm>

namespace gbfmm {

// ------------------------------------------------------------------------------------------
// Root box: min/max reduction with a non-finite check; the last block to finish folds the
// per-block partials and writes the box (no spin-wait: a completion counter elects it).
// ------------------------------------------------------------------------------------------
constexpr int kBoxThreads = 256;
constexpr int kBoxBlocks = 304;

__global__ void __launch_bounds__(kBoxThreads) k_bbox(const float4 *__restrict__ x, int64_t n, int has_box,
                                                      double ox, double oy, double oz, double bside, Box *box_out,
                                                      float *partials, unsigned *counter, int *status)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float4 p = __ldg(&x[i]);
        float c[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (isfinite(c[d])) {
                mn[d] = fminf(mn[d], c[d]);
                mx[d] = fmaxf(mx[d], c[d]);
            } else {
                bad = 1;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    bad = __any_sync(0xffffffffu, bad);
    __shared__ float red[kBoxThreads / 32][6];
    __shared__ int sbad;
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
            red[warp][d] = mn[d];
            red[warp][3 + d] = mx[d];
        }
        if (bad) atomicOr(&sbad, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float r[6];
        for (int k = 0; k < 6; ++k) r[k] = red[0][k];
        for (int w = 1; w < kBoxThreads / 32; ++w)
            for (int d = 0; d < 3; ++d) {
                r[d] = fminf(r[d], red[w][d]);
                r[3 + d] = fmaxf(r[3 + d], red[w][3 + d]);
            }
        for (int k = 0; k < 6; ++k) partials[blockIdx.x * 8 + k] = r[k];
        partials[blockIdx.x * 8 + 6] = sbad ? 1.f : 0.f;
        if (sbad) atomicOr(status, kStatusNonFinite);
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // fold the per-block partials with the whole block (strided loads, then a shuffle reduction)
    float r[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    int any_bad = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            r[d] = fminf(r[d], __ldcg(&partials[b * 8 + d]));
            r[3 + d] = fmaxf(r[3 + d], __ldcg(&partials[b * 8 + 3 + d]));
        }
        if (__ldcg(&partials[b * 8 + 6]) != 0.f) any_bad = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            r[d] = fminf(r[d], __shfl_xor_sync(0xffffffffu, r[d], o));
            r[3 + d] = fmaxf(r[3 + d], __shfl_xor_sync(0xffffffffu, r[3 + d], o));
        }
    any_bad = __any_sync(0xffffffffu, any_bad);
    __syncthreads();
    if (lane == 0) {
        for (int k = 0; k < 6; ++k) red[warp][k] = r[k];
        if (any_bad) atomicOr(&sbad, 2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBoxThreads / 32; ++w)
            for (int d = 0; d < 3; ++d) {
                r[d] = fminf(r[d], red[w][d]);
                r[3 + d] = fmaxf(r[3 + d], red[w][3 + d]);
            }
        any_bad = (sbad & 2) != 0;
        Box b;
        if (has_box) {
            b.origin[0] = ox;
            b.origin[1] = oy;
            b.origin[2] = oz;
            b.side = bside;
        } else if (n == 0 || any_bad || !(r[0] <= r[3])) {
            b.origin[0] = b.origin[1] = b.origin[2] = 0.0;
            b.side = 1.0;
        } else {
            double S = 0.0;
            for (int d = 0; d < 3; ++d) {
                double e = __dsub_rn((double)r[3 + d], (double)r[d]);
                if (e > S) S = e;
            }
            if (S == 0.0) S = 1.0;
            for (int d = 0; d < 3; ++d) {
                double c = __dmul_rn(__dadd_rn((double)r[d], (double)r[3 + d]), 0.5);
                b.origin[d] = __dsub_rn(c, __dmul_rn(S, 0.5));
            }
            b.side = S;
        }
        b.key_scale = __ddiv_rn(2097152.0, b.side);
        double m = 0.0;
        for (int d = 0; d < 3; ++d) {
            b.origin_f[d] = __double2float_rn(b.origin[d]);
            m = fmax(m, fabs(b.origin[d]));
        }
        b.key_scale_f = __double2float_rn(b.key_scale);
        b.key_scale_lo = __double2float_rn(__dsub_rn(b.key_scale, (double)b.key_scale_f));
        for (int d = 0; d < 3; ++d) b.origin_lo[d] = __double2float_rn(__dsub_rn(b.origin[d], (double)b.origin_f[d]));
        // twice the bound 2^-22 (|o| s + |v|) + 2^-40 of the FP32 estimate's error (see k_keys)
        b.key_slack = __double2float_ru(__dmul_ru(__dmul_ru(m, b.key_scale), 0x1p-21) + 0x1p-20);
        *box_out = b;
        *counter = 0u;  // ready for the next launch on this stream
    }
}

void launch_bbox(const float4 *x, int64_t n, int has_box, const double *box_origin, double box_side, Box *box_out,
                 float *partials, unsigned *counter, int *status, cudaStream_t s)
{
    int64_t want = (n + kBoxThreads - 1) / kBoxThreads;
    int blocks = (int)(want < kBoxBlocks ? (want > 0 ? want : 1) : kBoxBlocks);
    k_bbox<<<blocks, kBoxThreads, 0, s>>>(x, n, has_box, box_origin[0], box_origin[1], box_origin[2], box_side,
                                          box_out, partials, counter, status);
    note_launches(1);
}

// ------------------------------------------------------------------------------------------
// Morton keys at the leaf depth L: k_d = clamp(floor((x_d - origin_d) * s), 0, 2^21-1) with
// s = 2^21 / side (one IEEE FP64 division, in the box kernel), every step one IEEE FP64
// rounding; then the 3L-bit key of the depth-L cell = interleave(k_d >> (21 - L)).
// ------------------------------------------------------------------------------------------
//
// The uniform tree needs only the top L bits of each k_d, and those are found in FP32 for all
// but the particles within a few grid units of a leaf-cell face.  With o_f, s_f the FP32
// roundings of origin and scale, the estimate v_f = (x - o_f) s_f (two FP32 roundings) is
// within 2^-22 (|o| s + |v_f|) + 2^-40 of the FP64 value v, so v lies in [v_f - e, v_f + e]
// with e = |v_f| 2^-21 + key_slack (twice that bound).  The leaf index clamp(floor(v), 0,
// 2^21 - 1) >> (21 - L) is monotone in v: where it agrees at both ends of the interval it is
// the FP64 result; otherwise the particle takes the FP64 steps above.
GB_DEV uint32_t leaf_coord_f(float v, int sh)
{
    float f = floorf(v);
    if (!(f >= 0.f)) f = 0.f;  // also maps NaN to 0
    if (f > 2097151.f) f = 2097151.f;
    return (uint32_t)f >> sh;
}


__global__ void k_keys(const float4 *__restrict__ x, int64_t n, const Box *__restrict__ box, int L,
                       uint32_t *__restrict__ leafkey, uint32_t *__restrict__ idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Box b = *box;
    float4 p = __ldg(&x[i]);
    float c[3] = {p.x, p.y, p.z};
    const int sh = 21 - L;
    uint32_t k[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float vf = __fmul_rn(__fsub_rn(c[d], b.origin_f[d]), b.key_scale_f);
        const float e = __fadd_ru(__fmul_ru(fabsf(vf), 0x1p-21f), b.key_slack);
        const uint32_t lo = leaf_coord_f(__fsub_rd(vf, e), sh), hi = leaf_coord_f(__fadd_ru(vf, e), sh);
        k[d] = lo == hi ? lo : grid_coord_fp64(c[d], b.origin[d], b.key_scale) >> sh;
    }
    leafkey[i] = morton3(k[0], k[1], k[2]);
    idx[i] = (uint32_t)i;
}

void launch_keys(const float4 *x, int64_t n, const Box *box, int L, uint32_t *leafkey, uint32_t *idx, cudaStream_t s)
{
    if (n <= 0) return;
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, box, L, leafkey, idx);
    note_launches(1);
}

// ------------------------------------------------------------------------------------------
// Exclusive scan of uint32 (reduce, scan of block sums, apply).  out[n] receives the total.
// ------------------------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

size_t exclusive_scan_tmp_words(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                              uint32_t *__restrict__ part)
{
    int64_t base = blockIdx.x * (int64_t)kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        int64_t i = base + r * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// single block: exclusive scan of the nb block sums in place; total to *total
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *part, int64_t nb, uint32_t *total)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        uint32_t v = (i < nb) ? part[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = ws[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            ws[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        uint32_t c = carry;
        if (i < nb) part[i] = c + ws[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + ws[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *in, uint32_t *out, int64_t n,
                                                             const uint32_t *__restrict__ part)
{
    __shared__ uint32_t tile[kScanTile];
    __shared__ uint32_t ws[kScanThreads / 32];
    int64_t base = blockIdx.x * (int64_t)kScanTile;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        int64_t i = base + r * kScanThreads + threadIdx.x;
        tile[r * kScanThreads + threadIdx.x] = (i < n) ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t loc[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = s;
        s += tile[threadIdx.x * kScanItems + k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += ws[w];
    uint32_t pre = part[blockIdx.x] + wpre + incl - s;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = pre + loc[k];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        int64_t i = base + r * kScanThreads + threadIdx.x;
        if (i < n) out[i] = tile[r * kScanThreads + threadIdx.x];
    }
}

void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return;
    }
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb, out + n);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    note_launches(3);
}

// ------------------------------------------------------------------------------------------
// Stable LSD radix sort of (key, index) pairs, 8-bit digits: one kernel counts every digit
// position's histogram, then one kernel per digit position ranks and scatters the keys.
// Tiles of 4096 keys are taken in launch order (a counter), each ranks its keys stably in
// shared memory (per-warp counts over a blocked layout, warp match within a round), publishes
// its per-digit count and looks back over the earlier tiles' counts (decoupled look-back: an
// earlier tile publishes its count at once and its inclusive prefix when it has one) to find
// where its keys of each digit start.  The keys are staged in shared memory in tile-sorted
// order and written out in runs per digit.  The last pass also gathers the particles.
// Scratch: per-pass tile counters, the digit histograms, and one 64-bit status word per
// (pass, tile, digit): flag (bits 62-63: 1 = count, 2 = inclusive prefix) | value.
// ------------------------------------------------------------------------------------------
constexpr int kRsThreads = 512, kRsItems = 8, kRsTile = kRsThreads * kRsItems;  // tile of 4096 keys
constexpr int kRsWarps = kRsThreads / 32, kRsWarpKeys = kRsTile / kRsWarps;
constexpr int kRsHistThreads = 256;  // one per digit
constexpr int64_t kRsScanMinN = int64_t(1) << 22;  // from here on the passes take the reduce-then-scan form
constexpr uint64_t kRsAgg = 1ull << 62, kRsInc = 2ull << 62, kRsFlags = 3ull << 62;

static_assert(kRsWarpKeys == 32 * kRsItems, "blocked layout: a warp owns kRsItems rounds of 32 keys");
static_assert(kRsTile <= 65535, "16-bit per-warp digit counts and offsets");

GB_DEV void st_release_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

GB_DEV uint64_t ld_acquire_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

GB_DEV uint64_t timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// exclusive scan of one value per thread over the block (wsum: one word per warp)
GB_DEV uint32_t block_excl_scan(uint32_t v, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    __syncthreads();
    return off + x - v;
}

template <class KeyT>
__global__ void __launch_bounds__(kRsHistThreads) k_rs_ghist(const KeyT *__restrict__ keys, int64_t n, int passes,
                                                             uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t h[sizeof(KeyT)][256];
    for (int d = 0; d < passes; ++d) h[d][threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kRsHistThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kRsHistThreads) {
        const KeyT k = keys[i];
        for (int d = 0; d < passes; ++d) atomicAdd(&h[d][(uint32_t)(k >> (8 * d)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int d = 0; d < passes; ++d)
        if (h[d][threadIdx.x]) atomicAdd(&ghist[d * 256 + threadIdx.x], h[d][threadIdx.x]);
}

// LB: the tile's digit starts by decoupled look-back over the earlier tiles (tiles taken in
// launch order from a counter); else read from `starts` (tile_starts of the reduce-then-scan
// form: starts[d * nblk + tile]), tile = blockIdx.x
template <class KeyT, bool LB>
__global__ void __launch_bounds__(kRsThreads, 3) k_rs_pass(const KeyT *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                        KeyT *__restrict__ kout, uint32_t *__restrict__ vout,
                                                        int64_t n, int pass, int64_t nblk,
                                                        const uint32_t *__restrict__ ghist, uint64_t *status,
                                                        uint32_t *counter, const float4 *__restrict__ gx,
                                                        float4 *__restrict__ gsx, int *err,
                                                        const uint32_t *__restrict__ starts)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    KeyT *skey = reinterpret_cast<KeyT *>(rs_smem);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kRsTile);
    __shared__ uint16_t wcnt[kRsWarps][256];  // per-warp digit counts, then offsets (< kRsTile)
    __shared__ uint32_t dstart[256], gbase[256], wsum[kRsWarps];
    __shared__ uint32_t tile_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int shift = 8 * pass;
    const bool dig = tid < 256;  // the per-digit work: thread tid, digit tid
    if (tid == 0) tile_sh = LB ? atomicAdd(&counter[pass], 1u) : blockIdx.x;
    for (int e = tid; e < kRsWarps * 256; e += kRsThreads) (&wcnt[0][0])[e] = 0;
    __syncthreads();
    const int64_t tile = tile_sh;
    const int64_t base = tile * kRsTile + (int64_t)warp * kRsWarpKeys;
    // only the ranks stay in registers across the scans: the keys and indices are read again
    // (from L1 / L2) when they are staged, which leaves room for three CTAs per SM
    uint32_t rk[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {  // the digits first: all the warp's loads in flight at once
        const int64_t i = base + 32 * r + lane;
        rk[r] = i < n ? ((uint32_t)(kin[i] >> shift) & 0xffu) : 256u;
    }
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const uint32_t d = rk[r];
        const bool valid = d < 256u;
        // the lanes holding the same digit (invalid lanes: digit 256, a class of their own),
        // from one ballot per digit bit
        unsigned peers = __ballot_sync(0xffffffffu, valid);
        if (!valid) peers = ~peers;
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
            const unsigned bb = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bb : ~bb;
        }
        const uint32_t before = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        rk[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // digit tid: offsets of the warps' runs inside the tile's run, and the tile's count
    uint32_t cnt = 0;
    if (dig) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t t = wcnt[w][tid];
            wcnt[w][tid] = (uint16_t)cnt;
            cnt += t;
        }
    }
    const uint32_t ds = block_excl_scan(cnt, wsum);  // threads >= 256 add zeros after the digits
    if (dig) dstart[tid] = ds;
    if (!LB) {
        if (dig) gbase[tid] = starts[(int64_t)tid * nblk + tile];
    } else {
    // look back over the earlier tiles' counts of digit tid
    uint64_t *st = status + (size_t)pass * nblk * 256;
    uint32_t excl = 0;
    if (!dig) {
    } else if (tile == 0) {
        st_release_u64(&st[tid], kRsInc | cnt);
    } else {
        st_release_u64(&st[tile * 256 + tid], kRsAgg | cnt);
        const uint64_t t0 = timer_ns();
        for (int64_t t = tile - 1; t >= 0;) {
            const uint64_t w = ld_acquire_u64(&st[t * 256 + tid]);
            if ((w & kRsFlags) == 0) {
                if (timer_ns() - t0 > 1000000000ull) {  // 1 s: report and give up
                    atomicOr(err, kStatusTimeout);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl += (uint32_t)w;
            if ((w & kRsFlags) == kRsInc) break;
            --t;
        }
        st_release_u64(&st[tile * 256 + tid], kRsInc | (excl + cnt));
    }
    const uint32_t gb = block_excl_scan(dig ? ghist[pass * 256 + tid] : 0u, wsum);
    if (dig) gbase[tid] = gb + excl;
    }
    __syncthreads();
    // stage in tile-sorted order, then write the runs of each digit
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = base + 32 * r + lane;
        if (i < n) {
            const KeyT key = kin[i];
            const uint32_t d = (uint32_t)(key >> shift) & 0xffu;
            const uint32_t pos = dstart[d] + wcnt[warp][d] + rk[r];
            skey[pos] = key;
            sval[pos] = vin[i];
        }
    }
    __syncthreads();
    const int64_t t0 = tile * kRsTile;
    const int tn = (int)(n - t0 < kRsTile ? n - t0 : kRsTile);
    for (int jj = tid; jj < tn; jj += kRsThreads) {
        const KeyT key = skey[jj];
        const uint32_t val = sval[jj];
        const uint32_t d = (uint32_t)(key >> shift) & 0xffu;
        const uint32_t gp = gbase[d] + (uint32_t)jj - dstart[d];
        kout[gp] = key;
        vout[gp] = val;
        if (gsx) gsx[gp] = __ldg(&gx[val]);
    }
}

// Reduce-then-scan form of a pass (large inputs): every tile's digit counts (k_rs_upsweep),
// their exclusive scan in digit-major order started at each digit's global start
// (k_rs_tile_starts), then k_rs_pass<KeyT, false> ranks and scatters with those starts.  The
// passes then carry no chain from tile to tile (the look-back's latency bound the one-sweep
// passes on large inputs), for one more read of the keys per pass.
template <class KeyT>
__global__ void __launch_bounds__(256) k_rs_upsweep(const KeyT *__restrict__ kin, int64_t n, int pass, int64_t nblk,
                                                    uint32_t *__restrict__ counts)
{
    // one digit histogram per warp; a key is one shared-memory add (the whole warp's 32 in one
    // add when its lanes agree), not a ballot match per key: counting needs no ranks
    __shared__ uint32_t h[8][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k][tid] = 0;
    __syncthreads();
    const int64_t t0 = blockIdx.x * (int64_t)kRsTile;
    const int shift = 8 * pass;
    constexpr int R = kRsTile / 256;
    uint32_t dd[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {  // all the tile's loads in flight at once
        const int64_t i = t0 + r * 256 + tid;
        dd[r] = i < n ? ((uint32_t)(kin[i] >> shift) & 0xffu) : 256u;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t d = dd[r], d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, d == d0)) {
            if (lane == 0 && d0 < 256u) atomicAdd(&h[warp][d0], 32u);
        } else if (d < 256u) {
            atomicAdd(&h[warp][d], 1u);
        }
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) c += h[k][tid];
    counts[(int64_t)tid * nblk + blockIdx.x] = c;
}

// CTA d: starts[d * nblk + t] = (keys of digits < d) + (keys of digit d in tiles < t)
__global__ void __launch_bounds__(1024) k_rs_tile_starts(const uint32_t *__restrict__ counts,
                                                         uint32_t *__restrict__ starts, int64_t nblk,
                                                         const uint32_t *__restrict__ ghist, int pass)
{
    __shared__ uint32_t wsum[32], s_carry;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        uint32_t b = 0;
        for (int e = lane; e < d; e += 32) b += ghist[pass * 256 + e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (lane == 0) s_carry = b;
    }
    __syncthreads();
    const uint32_t *c = counts + (int64_t)d * nblk;
    uint32_t *o = starts + (int64_t)d * nblk;
    for (int64_t c0 = 0; c0 < nblk; c0 += 4 * 1024) {
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t t = c0 + 4 * tid + k;
            v[k] = t < nblk ? c[t] : 0u;
            sum += v[k];
        }
        const uint32_t carry = s_carry;
        const uint32_t ex = block_excl_scan(sum, wsum);
        uint32_t run = carry + ex;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t t = c0 + 4 * tid + k;
            if (t < nblk) o[t] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) s_carry = run;  // the chunk's end
        __syncthreads();
    }
}

__global__ void k_gather_identity(const float4 *__restrict__ x, float4 *__restrict__ sx, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) sx[i] = x[i];
}

template <class KeyT>
static void sort_gather_t(KeyT *k0, KeyT *k1, uint32_t *v0, uint32_t *v1, int64_t n, int bits, void *scratch,
                          int *err, const float4 *x, float4 *sx, KeyT **keys_out, uint32_t **idx_out,
                          cudaStream_t s)
{
    KeyT *kin = k0, *kout = k1;
    uint32_t *vin = v0, *vout = v1;
    if (bits <= 0 || n <= 1) {
        if (n > 0) {
            k_gather_identity<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, sx, n);
            note_launches(1);
        }
        *keys_out = k0;
        *idx_out = v0;
        return;
    }
    const int passes = (bits + 7) / 8;
    const int64_t nblk = (n + kRsTile - 1) / kRsTile;
    unsigned char *sc = static_cast<unsigned char *>(scratch);
    uint32_t *counter = reinterpret_cast<uint32_t *>(sc);
    uint32_t *ghist = reinterpret_cast<uint32_t *>(sc + kRsCounterBytes);
    uint64_t *status = reinterpret_cast<uint64_t *>(sc + kRsCounterBytes + kRsHistBytes);
    // large inputs of several passes take the reduce-then-scan form; its tile counts and starts
    // (4 bytes each per tile and digit) use the look-back words' space of the first two passes
    const bool rts = passes >= 2 && n >= kRsScanMinN;
    uint32_t *counts = reinterpret_cast<uint32_t *>(status);
    uint32_t *starts = counts + 256 * nblk;
    cudaMemsetAsync(scratch, 0, rts ? kRsCounterBytes + kRsHistBytes : sort_scratch_bytes(n, bits), s);
    const unsigned hgrid = (unsigned)std::min<int64_t>(nblk * (kRsTile / kRsHistThreads) / 4 + 1, 1216);
    k_rs_ghist<KeyT><<<hgrid, kRsHistThreads, 0, s>>>(kin, n, passes, ghist);
    const int smem = kRsTile * (int)(sizeof(KeyT) + sizeof(uint32_t));
    cudaFuncSetAttribute(k_rs_pass<KeyT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_rs_pass<KeyT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    for (int pass = 0; pass < passes; ++pass) {
        const bool last = pass + 1 == passes;
        if (rts) {
            k_rs_upsweep<KeyT><<<(unsigned)nblk, 256, 0, s>>>(kin, n, pass, nblk, counts);
            k_rs_tile_starts<<<256, 1024, 0, s>>>(counts, starts, nblk, ghist, pass);
            k_rs_pass<KeyT, false><<<(unsigned)nblk, kRsThreads, smem, s>>>(
                kin, vin, kout, vout, n, pass, nblk, ghist, status, counter, x, last ? sx : nullptr, err, starts);
            note_launches(2);
        } else {
            k_rs_pass<KeyT, true><<<(unsigned)nblk, kRsThreads, smem, s>>>(
                kin, vin, kout, vout, n, pass, nblk, ghist, status, counter, x, last ? sx : nullptr, err, nullptr);
        }
        KeyT *t = kin;
        kin = kout;
        kout = t;
        uint32_t *u = vin;
        vin = vout;
        vout = u;
    }
    note_launches(1 + passes);
    *keys_out = kin;
    *idx_out = vin;
}

void launch_sort_gather(uint32_t *k0, uint32_t *k1, uint32_t *v0, uint32_t *v1, int64_t n, int bits, void *scratch,
                        int *err, const float4 *x, float4 *sx, uint32_t **keys_out, uint32_t **idx_out,
                        cudaStream_t s)
{
    sort_gather_t<uint32_t>(k0, k1, v0, v1, n, bits, scratch, err, x, sx, keys_out, idx_out, s);
}

void launch_sort_gather64(uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, int64_t n, int bits,
                          void *scratch, int *err, const float4 *x, float4 *sx, uint64_t **keys_out,
                          uint32_t **idx_out, cudaStream_t s)
{
    sort_gather_t<uint64_t>(k0, k1, v0, v1, n, bits, scratch, err, x, sx, keys_out, idx_out, s);
}

// ------------------------------------------------------------------------------------------
// Cells: for every level, the first and one-past-last sorted position of each nonempty cell
// (arrays zeroed beforehand, so empty cells read begin == end == 0).
// ------------------------------------------------------------------------------------------
__global__ void k_cells(const uint32_t *__restrict__ sk, int64_t n, int L, int32_t *__restrict__ begin,
                        int32_t *__restrict__ end)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = sk[i];
    uint32_t prev = i > 0 ? sk[i - 1] : 0u, next = i + 1 < n ? sk[i + 1] : 0u;
    for (int l = 0; l <= L; ++l) {
        int sh = 3 * (L - l);
        uint32_t pk = key >> sh;
        int64_t g = level_offset(l) + pk;
        if (i == 0 || (prev >> sh) != pk) begin[g] = (int32_t)i;
        if (i + 1 == n || (next >> sh) != pk) end[g] = (int32_t)(i + 1);
    }
}

void launch_cells(const uint32_t *sk, int64_t n, int L, int32_t *begin, int32_t *end, cudaStream_t s)
{
    size_t C = (size_t)level_offset(L + 1);
    cudaMemsetAsync(begin, 0, C * sizeof(int32_t), s);
    cudaMemsetAsync(end, 0, C * sizeof(int32_t), s);
    if (n > 0) {
        k_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sk, n, L, begin, end);
        note_launches(1);
    }
}

// ------------------------------------------------------------------------------------------
// Interaction lists (Section "The P2P kernel implementation": 27 neighbour cells; Section
// "The M2L kernel implementation": at most 189 well-separated cells).
//   P2P row of a nonempty leaf: nonempty leaves at Chebyshev index distance <= 1 (itself
//       included), in ascending offset code (dz, dy, dx);
//   M2L row of a nonempty cell at level >= 2: nonempty children of the parent's neighbours
//       that are not neighbours themselves, in ascending offset code; the code
//       (dx+3) + 7(dy+3) + 49(dz+3) of the offset source - target is stored beside the id.
// ------------------------------------------------------------------------------------------
GB_DEV bool nonempty(const int32_t *begin, const int32_t *end, int64_t g) { return end[g] > begin[g]; }

GB_DEV void cell_of(int64_t g, int &l, uint32_t &key)
{
    l = 0;
    while (level_offset(l + 1) <= g) ++l;
    key = (uint32_t)(g - level_offset(l));
}

// Warp per cell.  The lanes test the 6 x 6 x 6 box of candidate offsets around the parent's
// neighbourhood (M2L) and the 27 neighbours (P2P) 32 at a time; a ballot keeps the candidates
// in ascending stencil-code order (offset index = ox + 6 oy + 36 oz, with the box's corner at
// -2 - (child bit)), the order the M2L kernels walk.
constexpr int kListWarps = 8;

// M2L = false: P2P rows only (the launch covers the leaf level, g0 = level_offset(L))
template <bool FILL, bool M2L = true>
__global__ void __launch_bounds__(32 * kListWarps) k_lists(int L, int64_t g0, int64_t C, const int32_t *__restrict__ begin,
                                                           const int32_t *__restrict__ end,
                                                           uint32_t *__restrict__ p2p_len, uint32_t *__restrict__ m2l_len,
                                                           const uint32_t *__restrict__ p2p_offs,
                                                           int32_t *__restrict__ p2p_ids,
                                                           const uint32_t *__restrict__ m2l_offs,
                                                           int32_t *__restrict__ m2l_ids, uint16_t *__restrict__ m2l_code)
{
    const int lane = threadIdx.x & 31;
    const int64_t g = g0 + blockIdx.x * (int64_t)kListWarps + (threadIdx.x >> 5);
    if (g >= C) return;
    int l;
    uint32_t key;
    cell_of(g, l, key);
    const bool ne = nonempty(begin, end, g);
    int x, y, z;
    demorton3(key, x, y, z);
    const int side = 1 << l;
    const int64_t off = level_offset(l);
    const unsigned lt = (1u << lane) - 1u;
    if (M2L && l >= 2) {
        uint32_t cnt = 0, e = FILL ? m2l_offs[g] : 0u;
        if (ne) {
            // all seven rounds' candidates first, so that their begin/end loads are in flight
            // together, then the ballots in order
            constexpr int kRounds = (216 + 31) / 32;
            const int bx = -2 - (x & 1), by = -2 - (y & 1), bz = -2 - (z & 1);
            int32_t src[kRounds];
            bool ok[kRounds];
#pragma unroll
            for (int r = 0; r < kRounds; ++r) {
                const int i = 32 * r + lane;
                const int ox = bx + i % 6, oy = by + (i / 6) % 6, oz = bz + i / 36;
                const int sx = x + ox, sy = y + oy, sz = z + oz;
                ok[r] = i < 216 && sx >= 0 && sy >= 0 && sz >= 0 && sx < side && sy < side && sz < side &&
                        !(ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1);
                src[r] = ok[r] ? (int32_t)(off + morton3((uint32_t)sx, (uint32_t)sy, (uint32_t)sz)) : 0;
            }
            int32_t b[kRounds], en[kRounds];
#pragma unroll
            for (int r = 0; r < kRounds; ++r) {
                b[r] = ok[r] ? __ldg(&begin[src[r]]) : 0;
                en[r] = ok[r] ? __ldg(&end[src[r]]) : 0;
            }
#pragma unroll
            for (int r = 0; r < kRounds; ++r) {
                const bool hit = ok[r] && en[r] > b[r];
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (FILL && hit) {
                    const int i = 32 * r + lane;
                    const uint32_t at = e + cnt + __popc(m & lt);
                    m2l_ids[at] = src[r];
                    m2l_code[at] = (uint16_t)gbfmm::m2l_code(bx + i % 6, by + (i / 6) % 6, bz + i / 36);
                }
                cnt += __popc(m);
            }
        }
        if (!FILL && lane == 0) m2l_len[g] = cnt;
    } else if (M2L && !FILL && lane == 0) {
        m2l_len[g] = 0;
    }
    if (l == L) {
        uint32_t cnt = 0, e = FILL ? p2p_offs[key] : 0u;
        if (ne) {
            const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
            const int sx = x + ox, sy = y + oy, sz = z + oz;
            bool ok = lane < 27 && sx >= 0 && sy >= 0 && sz >= 0 && sx < side && sy < side && sz < side;
            int64_t s = 0;
            if (ok) {
                s = off + morton3((uint32_t)sx, (uint32_t)sy, (uint32_t)sz);
                ok = nonempty(begin, end, s);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (FILL && ok) p2p_ids[e + __popc(m & lt)] = (int32_t)s;
            cnt = __popc(m);
        }
        if (!FILL && lane == 0) p2p_len[key] = cnt;
    }
}

void launch_list_count(int L, const int32_t *begin, const int32_t *end, uint32_t *p2p_len, uint32_t *m2l_len,
                       cudaStream_t s)
{
    const int64_t C = level_offset(L + 1);
    k_lists<false><<<(unsigned)((C + kListWarps - 1) / kListWarps), 32 * kListWarps, 0, s>>>(
        L, 0, C, begin, end, p2p_len, m2l_len, nullptr, nullptr, nullptr, nullptr, nullptr);
    note_launches(1);
}

void launch_p2p_list_count(int L, const int32_t *begin, const int32_t *end, uint32_t *p2p_len, cudaStream_t s)
{
    const int64_t g0 = level_offset(L), C = level_offset(L + 1);
    k_lists<false, false><<<(unsigned)((C - g0 + kListWarps - 1) / kListWarps), 32 * kListWarps, 0, s>>>(
        L, g0, C, begin, end, p2p_len, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    note_launches(1);
}

void launch_p2p_list_fill(int L, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs, int32_t *p2p_ids,
                          cudaStream_t s)
{
    const int64_t g0 = level_offset(L), C = level_offset(L + 1);
    k_lists<true, false><<<(unsigned)((C - g0 + kListWarps - 1) / kListWarps), 32 * kListWarps, 0, s>>>(
        L, g0, C, begin, end, nullptr, nullptr, p2p_offs, p2p_ids, nullptr, nullptr, nullptr);
    note_launches(1);
}

void launch_list_fill(int L, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs, int32_t *p2p_ids,
                      const uint32_t *m2l_offs, int32_t *m2l_ids, uint16_t *m2l_code, cudaStream_t s)
{
    const int64_t C = level_offset(L + 1);
    k_lists<true><<<(unsigned)((C + kListWarps - 1) / kListWarps), 32 * kListWarps, 0, s>>>(
        L, 0, C, begin, end, nullptr, nullptr, p2p_offs, p2p_ids, m2l_offs, m2l_ids, m2l_code);
    note_launches(1);
}

}  // namespace gbfmm
