// M2L (Eq. 4) of the uniform tree as a block convolution on the tcgen05 tensor cores.
//
// On the uniform tree the M2L list of a level-l cell t = 2Q + tau (Q its parent's integer
// coordinates, tau its child position) holds the children sigma of the parent's 26 neighbours
// S = Q + D whose offset o = 2D + sigma - tau is not a near neighbour (|o|_inf >= 2).  Grouped by
// the parent offset D, the M2L of all 8 children of Q is
//     L~(Q, tau) = sum_D sum_sigma B_D[tau][sigma] M~(Q + D, sigma),
//     B_D[tau][sigma] = T_{2D + sigma - tau} if |2D + sigma - tau|_inf >= 2, else 0,
// where T_o is the p^2 x p^2 real M2L operator of offset o (Eq. 4-6, scaled expansions).  Over
// the parents of a level this is one dense GEMM per D:
//     D[Q][(tau, n)] += sum_(sigma, k) A[Q + D][(sigma, k)] B_D[(tau, n)][(sigma, k)],
// A[S] = the 8 p^2 multipole coefficients of the children of parent S (zero for empty cells and
// for S outside the level).  K = N = 8 p^2 (800 at p = 10): no padding, and the zero blocks of
// B_D (near pairs) are 9% of its entries.  No interaction lists are read.
//
// Tiles: one CTA takes 128 target parents (a box of 8 x 4 x 4 in the parent grid; smaller on
// levels 2 and 3) as the MMA's M and one N-tile of the 8 p^2 outputs, and walks the 26 offsets
// D in chunks of 32 or 64 K values.  Operands stream through shared memory by TMA tiled loads
// (the source box shifted by D, out-of-range parents zero-filled; B_D's N-tile), swizzled,
// and both are read by the MMA from shared memory.  Precision is the 3xF16 scheme of the
// gathered kernel: x = hi + lo in FP16, D += A_lo B_hi + A_hi B_lo + A_hi B_hi with FP32
// accumulation in TMEM.  Scales: every source parent's coefficients by 2^s_S (max -> 2^10), the
// operators by one power of two 2^g (max over all offsets -> 2^12).  Each D's partial is drained
// from TMEM (in DS pieces along K, bounding the truncating accumulation chain) to FP32 registers
// and multiplied by 2^-(s_(Q+D) + g) per row before the sum; two TMEM accumulators alternate so
// the MMAs of the next piece overlap the drain.
#include "common.cuh"
#include "ptx.cuh"

#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

namespace gbfmm {

namespace {

constexpr int kBlkRows = 128;  // target parents per CTA (MMA M)
constexpr int kBlkDrainWarps = 8;
// drains per offset: each offset's K range (8 p^2) is accumulated in TMEM in two pieces, so no
// truncating accumulation chain is longer than about half an offset (75 MMAs at p = 10)
constexpr int kBlkDrainsPerOffset = 2;
constexpr int kBlkThreads = 32 * (kBlkDrainWarps + 2);  // drain warps, TMA producer, MMA issuer

// the 26 parent offsets D in {-1, 0, 1}^3 \ {0}: index d -> D
GB_HD void blk_delta(int d, int &dx, int &dy, int &dz)
{
    const int i = d < 13 ? d : d + 1;
    dx = i % 3 - 1;
    dy = (i / 3) % 3 - 1;
    dz = i / 9 - 1;
}

}  // namespace

// CH: K values per pipeline stage, one swizzled shared-memory row (64: 128-byte swizzle, 32:
// 64-byte swizzle)
template <int P, int CH>
struct BlkCfg {
    static constexpr int PP = P * P, KD = 8 * PP;
    // N-tile: rows of B_D per CTA (the MMA's N, a multiple of 16) and the stride between tiles
    static constexpr int NT = P == 4 ? 128 : P == 6 ? 144 : P == 8 ? 256 : 208;
    static constexpr int NSTRIDE = P == 10 ? 200 : NT;
    static constexpr int NTILES = (KD + NSTRIDE - 1) / NSTRIDE;
    static constexpr int NKC = (KD + CH - 1) / CH;
    static constexpr int A_BYTES = kBlkRows * CH * 2;  // one of hi / lo
    static constexpr int B_BYTES = NT * CH * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int NSTAGE_FIT = (210 * 1024) / STAGE_BYTES;
    static constexpr int NSTAGE = NSTAGE_FIT > 4 ? 4 : NSTAGE_FIT;
    static constexpr size_t kSmemBytes = (size_t)NSTAGE * STAGE_BYTES + 1024;  // + alignment slack
    static constexpr int NH = NT / 2;  // accumulator columns per drain thread
    static constexpr int TMEM_COLS = 2 * NT <= 256 ? 256 : 512;
    static_assert(NT % 16 == 0 && NT <= 256, "MMA N");
    static_assert(NH % 8 == 0 && NSTRIDE % 4 == 0 && PP % 4 == 0, "drain / store granularity");
    static_assert(NSTRIDE <= NT && NTILES * NSTRIDE >= KD, "N tiling");
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzle atoms");
    static_assert(CH == 64 || CH == 32, "swizzled row of 128 or 64 bytes");
    static_assert(NSTAGE >= 2, "pipeline stages");
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};

// tensor maps and tiling of one launch (kernel parameter, read by the TMA unit in place)
struct BlkParams {
    CUtensorMap tmA[kMaxLevel + 1];  // per target level l: the presplit sources of the level's children
    CUtensorMap tmB;                 // B_D, FP16 hi | lo
    int L;
    int tile_lo[kMaxLevel + 2];      // tiles of level l: [tile_lo[l], tile_lo[l + 1]) (levels in ascending order)
    int tile0;                       // tile of block 0 (launch in waves)
    int ksplit;                      // the 26 offsets are split into ksplit ranges, one per CTA
    int64_t part_stride;             // ksplit > 1: floats between the partial sums of two ranges
};

// ---- shared-memory matrix descriptor, K-major, swizzled -----------------------------------------
// rows of 2 CH bytes, 8-row atoms of 16 CH bytes (SBO); a K step of 16 halves advances the start
// address by 32 bytes inside the atom.  Swizzle mode: 2 = 128-byte, 4 = 64-byte.
template <int CH>
GB_DEV uint64_t blk_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                   // LBO (unused for swizzled K-major operands)
    d |= (uint64_t)((16 * CH) >> 4) << 32;    // SBO: 8-row atoms
    d |= (uint64_t)1 << 46;                   // descriptor version of the 5th-generation tensor cores
    d |= (uint64_t)(CH == 64 ? 2 : 4) << 61;  // swizzle mode
    return d;
}

GB_DEV void blk_mma_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

GB_DEV void blk_tma5(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3, int c4, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

GB_DEV void blk_tma4(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

GB_DEV void blk_prefetch_tmap(const CUtensorMap *tm)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// whole warp: 8 consecutive 32-bit columns of the thread's TMEM lane, no wait
GB_DEV void blk_ld8(uint32_t taddr, uint32_t *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// 2^e as a float (e within the normal range)
GB_DEV float blk_pow2(int e) { return __int_as_float((127 + e) << 23); }

// ---- pre-split sources: per parent S of level l - 1, in grid order (x fastest), the 8 p^2
// coefficients of its children (child sigma at [sigma p^2, (sigma + 1) p^2)) scaled by 2^s_S and
// split into FP16 hi (plane 0) and lo (plane 1); s_S = 10 - e with max |M~| = f 2^e, f in
// [0.5, 1) over the parent's nonempty children (empty children and empty parents: zeros, s = 0).
// One warp per parent.
template <int P>
__global__ void __launch_bounds__(256) k_blk_presplit(int l, const int32_t *__restrict__ begin,
                                                      const int32_t *__restrict__ end, const float *__restrict__ M,
                                                      __half *__restrict__ A, int8_t *__restrict__ scale)
{
    constexpr int PP = P * P, KD = 8 * PP, PER = (KD + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int lp = l - 1;
    const int64_t np = int64_t(1) << (3 * lp);
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= np) return;
    const int pg = 1 << lp;
    const int x = (int)(i % pg), y = (int)((i / pg) % pg), z = (int)(i / ((int64_t)pg * pg));
    const int64_t c0 = level_offset(l) + 8 * (int64_t)morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
    float v[PER];
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = lane + 32 * j;
        float a = 0.f;
        if (k < KD) {
            const int64_t c = c0 + k / PP;
            if (end[c] > begin[c]) a = M[c0 * PP + k];
        }
        v[j] = a;
        m = fmaxf(m, fabsf(a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const bool fin = m > 0.f && m <= 3.0e38f;
    int ex = 0;
    if (fin) frexpf(m, &ex);
    int sc = fin ? 10 - ex : 0;
    sc = sc < -100 ? -100 : (sc > 100 ? 100 : sc);
    if (lane == 0) scale[i] = (int8_t)sc;
    const float up = blk_pow2(sc);
    __half *row = A + i * (2 * KD);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = lane + 32 * j;
        if (k < KD) {
            const float xs = v[j] * up;
            const __half hi = __float2half_rn(xs);
            row[k] = hi;
            row[KD + k] = __float2half_rn(xs - __half2float(hi));
        }
    }
}

// ---- operator blocks B_D (FP16 hi | lo, scaled by 2^g) -----------------------------------------
// largest |entry| over the admissible offsets' operators, as float bits (non-negative floats
// order like their bit patterns)
template <int P>
__global__ void __launch_bounds__(256) k_blk_opmax(const float *__restrict__ ops, unsigned *__restrict__ mbits)
{
    constexpr int PP = P * P, PR = ops_rows_padded(P);
    const int code = blockIdx.x;
    const int ox = code % 7 - 3, oy = (code / 7) % 7 - 3, oz = code / 49 - 3;
    if (max(abs(ox), max(abs(oy), abs(oz))) < 2) return;  // near offsets have no M2L operator
    const float *src = ops + (size_t)code * PP * PR;
    float m = 0.f;
    for (int e = threadIdx.x; e < PP * PP; e += blockDim.x) m = fmaxf(m, fabsf(src[(e / PP) * PR + e % PP]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mbits, __float_as_uint(m));
}

// B[d][plane][row (tau, n)][col (sigma, k)], one block per (d, row); g stored after the table
template <int P>
__global__ void __launch_bounds__(256) k_blk_build(const float *__restrict__ ops, const unsigned *__restrict__ mbits,
                                                   __half *__restrict__ B, int *__restrict__ gout)
{
    constexpr int PP = P * P, PR = ops_rows_padded(P), KD = 8 * PP;
    const int d = blockIdx.x / KD, row = blockIdx.x % KD;
    const int tau = row / PP, n = row % PP;
    int dx, dy, dz;
    blk_delta(d, dx, dy, dz);
    int ex = 0;
    const float m = __uint_as_float(*mbits);
    if (m > 0.f) frexpf(m, &ex);
    const int g = m > 0.f ? 12 - ex : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *gout = g;
    const float sc = blk_pow2(g);
    __half *hi = B + ((size_t)d * 2 * KD + row) * KD;
    __half *lo = hi + (size_t)KD * KD;
    for (int col = threadIdx.x; col < KD; col += blockDim.x) {
        const int sigma = col / PP, k = col % PP;
        const int ox = 2 * dx + (sigma & 1) - (tau & 1), oy = 2 * dy + ((sigma >> 1) & 1) - ((tau >> 1) & 1),
                  oz = 2 * dz + (sigma >> 2) - (tau >> 2);
        float v = 0.f;
        if (max(abs(ox), max(abs(oy), abs(oz))) >= 2)
            v = ops[(size_t)m2l_code(ox, oy, oz) * PP * PR + (size_t)k * PR + n] * sc;
        const __half h = __float2half_rn(v);
        hi[col] = h;
        lo[col] = __float2half_rn(v - __half2float(h));
    }
}

// ---- the kernel -------------------------------------------------------------------------------
template <int P, int DS, int CH>
__global__ void __launch_bounds__(kBlkThreads, 1)
    k_m2l_blk(const __grid_constant__ BlkParams prm, const int32_t *__restrict__ begin,
              const int32_t *__restrict__ end, const int8_t *__restrict__ pscale, const int *__restrict__ gexp,
              float *__restrict__ Lc, float *__restrict__ Lpart, int *status)
{
    using C = BlkCfg<P, CH>;
    constexpr int PP = C::PP, KD = C::KD, NT = C::NT, NH = C::NH, NKC = C::NKC, NSTAGE = C::NSTAGE;
    constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(kBlkRows >> 4) << 24);
    constexpr int kProdWarp = kBlkDrainWarps, kMmaWarp = kBlkDrainWarps + 1;

    extern __shared__ unsigned char blk_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], dfull[2], dempty[2], done_bar;
    __shared__ int s_issued[NSTAGE];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    // ---- tile: level, target parent box, N-tile; offset range [d_lo, d_hi)
    const int ks = (prm.tile0 + (int)blockIdx.x) % prm.ksplit;
    const int tile = (prm.tile0 + (int)blockIdx.x) / prm.ksplit;
    const int d_lo = (26 * ks) / prm.ksplit, d_hi = (26 * (ks + 1)) / prm.ksplit;
    const int S = (d_hi - d_lo) * NKC, NU = (d_hi - d_lo) * DS;
    int l = 2;
    while (l < prm.L && tile >= prm.tile_lo[l + 1]) ++l;
    const int pg = 1 << (l - 1);
    const int bx = pg < 8 ? pg : 8, by = pg < 4 ? pg : 4, bz = by;
    const int rows = bx * by * bz;
    int t = tile - prm.tile_lo[l];
    const int nt = t % C::NTILES;
    t /= C::NTILES;
    const int tx = t % (pg / bx), ty = (t / (pg / bx)) % (pg / by), tz = t / ((pg / bx) * (pg / by));
    const int x0 = tx * bx, y0 = ty * by, z0 = tz * bz;
    const uint32_t a_bytes = (uint32_t)rows * CH * 2;

    unsigned char *smem =
        blk_smem_raw + ((1024u - (smem_u32(blk_smem_raw) & 1023u)) & 1023u);  // 1024-byte aligned stages
    auto a_hi = [&](int st) { return smem + (size_t)st * C::STAGE_BYTES; };
    auto a_lo = [&](int st) { return smem + (size_t)st * C::STAGE_BYTES + C::A_BYTES; };
    auto b_hi = [&](int st) { return smem + (size_t)st * C::STAGE_BYTES + 2 * C::A_BYTES; };
    auto b_lo = [&](int st) { return smem + (size_t)st * C::STAGE_BYTES + 2 * C::A_BYTES + C::B_BYTES; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < NSTAGE; ++st) {
            mbar_init(&full_bar[st], 1);   // the producer's expect_tx arrival
            mbar_init(&empty_bar[st], 1);  // one tcgen05.commit
            s_issued[st] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], kBlkDrainWarps);
        }
        mbar_init(&done_bar, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == kProdWarp && lane == 0) {
        blk_prefetch_tmap(&prm.tmA[l]);
        blk_prefetch_tmap(&prm.tmB);
    }
    if (warp == kMmaWarp) tmem_alloc(&s_tmem, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // pipeline step s: offset d = s / NKC, K-chunk c = s % NKC; drain unit u = d DS + c DS / NKC
    if (warp == kProdWarp) {
        if (lane == 0) {
            for (int s = 0; s < S; ++s) {
                const int st = s % NSTAGE, d = d_lo + s / NKC, c = s % NKC;
                if (s >= NSTAGE &&
                    !mbar_wait_bounded(&empty_bar[st], ((s / NSTAGE) - 1) & 1, kWaitLimitNs, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                int dx, dy, dz;
                blk_delta(d, dx, dy, dz);
                mbar_expect_tx(&full_bar[st], 2u * a_bytes + 2u * (uint32_t)C::B_BYTES);
                const int k0 = c * CH;
                blk_tma5(a_hi(st), &prm.tmA[l], k0, 0, x0 + dx, y0 + dy, z0 + dz, &full_bar[st]);
                blk_tma5(a_lo(st), &prm.tmA[l], k0, 1, x0 + dx, y0 + dy, z0 + dz, &full_bar[st]);
                blk_tma4(b_hi(st), &prm.tmB, k0, nt * C::NSTRIDE, 0, d, &full_bar[st]);
                blk_tma4(b_lo(st), &prm.tmB, k0, nt * C::NSTRIDE, 1, d, &full_bar[st]);
                s_issued[st] += 1;
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            for (int s = 0; s < S; ++s) {
                const int st = s % NSTAGE, c = s % NKC;
                const int uc = (c * DS) / NKC, u = (s / NKC) * DS + uc, b = u & 1;
                const bool first = c == 0 || ((c - 1) * DS) / NKC != uc;
                const bool last = c == NKC - 1 || ((c + 1) * DS) / NKC != uc;
                if (first && u >= 2 &&
                    !mbar_wait_bounded(&dempty[b], ((u - 2) >> 1) & 1, kWaitLimitNs, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                if (!mbar_wait_bounded(&full_bar[st], (s / NSTAGE) & 1, kWaitLimitNs, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const int kw = KD - c * CH < CH ? KD - c * CH : CH;
                const uint32_t ah = smem_u32(a_hi(st)), al = smem_u32(a_lo(st));
                const uint32_t bh = smem_u32(b_hi(st)), bl = smem_u32(b_lo(st));
                const uint32_t dt = tmem + (uint32_t)(b * NT);
                for (int j = 0; j < (kw + 15) / 16; ++j) {
                    const uint32_t o = 32u * j;
                    blk_mma_ss(dt, blk_desc<CH>(al + o), blk_desc<CH>(bh + o), kIdesc, (first && j == 0) ? 0u : 1u);
                    blk_mma_ss(dt, blk_desc<CH>(ah + o), blk_desc<CH>(bl + o), kIdesc, 1u);
                    blk_mma_ss(dt, blk_desc<CH>(ah + o), blk_desc<CH>(bh + o), kIdesc, 1u);
                }
                tc_commit(&empty_bar[st]);
                if (last) tc_commit(&dfull[b]);
            }
            tc_commit(&done_bar);
        }
    } else {
        // ===== drain warps: row r (target parent), columns [h NH, h NH + NH) of the N-tile =====
        const int quad = warp & 3, h = warp >> 2;
        const int r = 32 * quad + lane;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        const bool rok = r < rows;
        const int qx = x0 + r % bx, qy = y0 + (r / bx) % by, qz = z0 + r / (bx * by);
        const int8_t *sl = pscale + (level_offset(l - 1) - 1);  // parents of level l - 1 (levels >= 1)
        const int g = *gexp;
        float acc[NH];
#pragma unroll
        for (int i = 0; i < NH; ++i) acc[i] = 0.f;
        bool alive = true;
        for (int u = 0; u < NU && alive; ++u) {
            const int d = d_lo + u / DS, b = u & 1;
            int dx, dy, dz;
            blk_delta(d, dx, dy, dz);
            const int sx = qx + dx, sy = qy + dy, sz = qz + dz;
            float f = 0.f;
            if (rok && sx >= 0 && sy >= 0 && sz >= 0 && sx < pg && sy < pg && sz < pg)
                f = blk_pow2(-((int)sl[sx + pg * (sy + pg * sz)] + g));
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&dfull[b], (u >> 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                alive = false;
                break;
            }
            tc_fence_after();
            const uint32_t col0 = tmem + lane_base + (uint32_t)(b * NT + h * NH);
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += 32) {
                constexpr int W = 32;
                uint32_t v[W];
#pragma unroll
                for (int q = 0; q < W; q += 8)
                    if (c0 + q < NH) blk_ld8(col0 + (uint32_t)(c0 + q), v + q);
                tmem_wait_ld_regs(v);
#pragma unroll
                for (int q = 0; q < W; ++q)
                    if (c0 + q < NH) acc[c0 + q] = fmaf(__uint_as_float(v[q]), f, acc[c0 + q]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[b]);
        }
        if (!alive && lane == 0) s_abort = 1;
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&done_bar, 0u, kWaitLimitNs, nullptr) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) s_abort = 1;
        __syncwarp();
        if (ok && alive && !s_abort && rok) {
            float *dst = prm.ksplit > 1 ? Lpart + (int64_t)ks * prm.part_stride : Lc;
            const int64_t cell0 = level_offset(l) + 8 * (int64_t)morton3((uint32_t)qx, (uint32_t)qy, (uint32_t)qz);
#pragma unroll
            for (int i = 0; i < NH; i += 4) {
                const int col = h * NH + i;
                const int gc = nt * C::NSTRIDE + col;
                if (col >= C::NSTRIDE || gc >= KD) continue;
                const int tau = gc / PP, n = gc % PP;
                const int64_t cell = cell0 + tau;
                if (end[cell] <= begin[cell]) continue;
                *reinterpret_cast<float4 *>(dst + cell * PP + n) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            atomicOr(status, kStatusTimeout);
            for (int st = 0; st < NSTAGE; ++st)
                if (s_issued[st] > 0) mbar_wait_bounded(&full_bar[st], (s_issued[st] - 1) & 1, kWaitLimitNs, nullptr);
        }
        __syncthreads();
    }
    if (warp == kMmaWarp) {
        __syncwarp();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// ---- the same block M2L on the adaptive tree ---------------------------------------------------
// On the adaptive tree the V list of a cell t (child tau of parent Q) is the children sigma of
// Q's colleagues S = Q + D (the positional colleagues of the level, D != 0) with |2D + sigma -
// tau|_inf >= 2: the block form above with S taken from the colleague table instead of the
// dense grid.  A colleague that is absent or a leaf, and a child that is absent, contribute zero
// coefficients; a colleague that is a leaf reaches t through its U or X list instead.  Target
// units are the cells of levels >= 1 with children (their children are the targets of levels
// >= 2), numbered in cell order; unit u has a row of the 8 p^2 coefficients of its children in
// the pre-split array (k_ablk_presplit), and row Z (the unit capacity) is zero.  A tile is 128
// consecutive units; its A operand for offset D gathers the rows of the units' colleagues
// (k_ablk_src: the row of every (unit, D), Z where the colleague has no children) by two loader
// warps (16-byte loads, stored in the swizzled layout the TMA writes for the dense form, then a
// proxy fence and one arrival each); B_D comes by TMA as before.

// unit numbering: flag of every cell (levels >= 1 with children)
__global__ void k_ablk_flags(Span cells, const int32_t *__restrict__ level, const int32_t *__restrict__ nchild,
                             uint32_t *__restrict__ flag)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cells.cap) return;
    uint32_t f = 0;
    if (i < span_count(cells)) {
        const int64_t c = span_first(cells) + i;
        f = (level[c] >= 1 && nchild[c] > 0) ? 1u : 0u;
    }
    flag[i] = f;
}

// unit_of[c] = its unit or -1; units[u] = its cell; n_units (one word) = the count
__global__ void k_ablk_units(Span cells, const uint32_t *__restrict__ flag, const uint32_t *__restrict__ scan,
                             int32_t *__restrict__ unit_of, int32_t *__restrict__ units, int32_t *__restrict__ n_units)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *n_units = (int32_t)scan[cells.cap];
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
    if (flag[i]) {
        unit_of[c] = (int32_t)scan[i];
        units[scan[i]] = (int32_t)c;
    } else {
        unit_of[c] = -1;
    }
}

// pre-split rows: unit u (one warp): its children's scaled coefficients 2^s_u M~ in FP16 hi | lo,
// s_u = 10 - e with max |M~| = f 2^e over its children (0 and zeros for none); row Z and its scale
// are zero
template <int P>
__global__ void __launch_bounds__(256) k_ablk_presplit(const int32_t *__restrict__ n_units, int64_t zrow,
                                                       const int32_t *__restrict__ units,
                                                       const int32_t *__restrict__ child_of,
                                                       const float *__restrict__ M, __half *__restrict__ A,
                                                       int8_t *__restrict__ scale)
{
    constexpr int PP = P * P, KD = 8 * PP, PER = (KD + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t u = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nu = *n_units;
    if (u > zrow || (u >= nu && u != zrow)) return;
    __half *row = A + u * (2 * KD);
    if (u == zrow || u >= nu) {
        for (int k = lane; k < 2 * KD; k += 32) row[k] = __float2half_rn(0.f);
        if (lane == 0) scale[u] = 0;
        return;
    }
    const int64_t q = units[u];
    float v[PER];
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = lane + 32 * j;
        float a = 0.f;
        if (k < KD) {
            const int32_t c = child_of[q * 8 + k / PP];
            if (c >= 0) a = M[(int64_t)c * PP + k % PP];
        }
        v[j] = a;
        m = fmaxf(m, fabsf(a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const bool fin = m > 0.f && m <= 3.0e38f;
    int ex = 0;
    if (fin) frexpf(m, &ex);
    int sc = fin ? 10 - ex : 0;
    sc = sc < -100 ? -100 : (sc > 100 ? 100 : sc);
    if (lane == 0) scale[u] = (int8_t)sc;
    const float up = blk_pow2(sc);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = lane + 32 * j;
        if (k < KD) {
            const float xs = v[j] * up;
            const __half hi = __float2half_rn(xs);
            row[k] = hi;
            row[KD + k] = __float2half_rn(xs - __half2float(hi));
        }
    }
}

// src[(tile 26 + d) 128 + r] = the row of unit tile 128 + r's colleague at offset d (Z if none);
// ucap: the units covered, a multiple of 128
__global__ void k_ablk_src(const int32_t *__restrict__ n_units, int64_t ucap, int64_t zrow,
                           const int32_t *__restrict__ units, const int32_t *__restrict__ coll,
                           const int32_t *__restrict__ unit_of, int32_t *__restrict__ src)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // over units (padded to tiles) x 26
    if (i >= ucap * 26) return;
    const int64_t u = i / 26;
    const int d = (int)(i % 26);
    int32_t row = (int32_t)zrow;
    if (u < *n_units) {
        int dx, dy, dz;
        blk_delta(d, dx, dy, dz);
        const int32_t s = coll[(int64_t)units[u] * 27 + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
        if (s >= 0 && unit_of[s] >= 0) row = unit_of[s];
    }
    src[((u / kBlkRows) * 26 + d) * kBlkRows + u % kBlkRows] = row;
}

constexpr int kAblkLoadWarps = 2;  // each loads 64 rows (more would leave the drains too few registers)
constexpr int kAblkThreads = 32 * (kBlkDrainWarps + kAblkLoadWarps + 2);  // drains, loaders, B producer, MMA

struct AblkParams {
    CUtensorMap tmB;  // B_D, FP16 hi | lo
    int tile0;        // tile of block 0 (launch in waves)
    int ksplit;
    int64_t part_stride;  // floats between the partial sums of two offset ranges
    int64_t zrow;
};

template <int P, int DS, int CH>
__global__ void __launch_bounds__(kAblkThreads, 1)
    k_m2l_ablk(const __grid_constant__ AblkParams prm, const int32_t *__restrict__ n_units,
               const int32_t *__restrict__ units, const int32_t *__restrict__ child_of,
               const int32_t *__restrict__ src, const __half *__restrict__ Apre, const int8_t *__restrict__ uscale,
               const int *__restrict__ gexp, float *__restrict__ Lc, float *__restrict__ Lpart, int *status)
{
    using C = BlkCfg<P, CH>;
    constexpr int PP = C::PP, KD = C::KD, NT = C::NT, NH = C::NH, NKC = C::NKC, NSTAGE = C::NSTAGE;
    constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(kBlkRows >> 4) << 24);
    constexpr int kLoad0 = kBlkDrainWarps, kProdWarp = kLoad0 + kAblkLoadWarps, kMmaWarp = kProdWarp + 1;

    extern __shared__ unsigned char blk_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], dfull[2], dempty[2], done_bar;
    __shared__ int s_issued[NSTAGE];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    // ---- tile: unit tile, N-tile, offset range [d_lo, d_hi)
    const int ks = (prm.tile0 + (int)blockIdx.x) % prm.ksplit;
    const int tt = (prm.tile0 + (int)blockIdx.x) / prm.ksplit;
    const int nt = tt % C::NTILES;
    const int64_t ut = tt / C::NTILES;
    const int64_t nu = *n_units;
    if (ut * kBlkRows >= nu) return;  // the whole CTA: past the units (before any barrier or TMEM)
    const int d_lo = (26 * ks) / prm.ksplit, d_hi = (26 * (ks + 1)) / prm.ksplit;
    const int S = (d_hi - d_lo) * NKC, NU = (d_hi - d_lo) * DS;
    const int32_t *tsrc = src + ut * 26 * kBlkRows;

    unsigned char *smem =
        blk_smem_raw + ((1024u - (smem_u32(blk_smem_raw) & 1023u)) & 1023u);  // 1024-byte aligned stages
    auto a_pl = [&](int st, int pl) { return smem + (size_t)st * C::STAGE_BYTES + pl * C::A_BYTES; };
    auto b_hi = [&](int st) { return smem + (size_t)st * C::STAGE_BYTES + 2 * C::A_BYTES; };
    auto b_lo = [&](int st) { return smem + (size_t)st * C::STAGE_BYTES + 2 * C::A_BYTES + C::B_BYTES; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < NSTAGE; ++st) {
            mbar_init(&full_bar[st], kAblkLoadWarps + 1);  // the loader warps + the B copies' expect_tx
            mbar_init(&empty_bar[st], 1);                  // one tcgen05.commit
            s_issued[st] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], kBlkDrainWarps);
        }
        mbar_init(&done_bar, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == kProdWarp && lane == 0) blk_prefetch_tmap(&prm.tmB);
    if (warp == kMmaWarp) tmem_alloc(&s_tmem, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp >= kLoad0 && warp < kProdWarp) {
        // ===== loader warps: rows 64 w + lane and 64 w + 32 + lane of A (hi and lo planes) =====
        // a stage's 16-byte chunks go through registers; where they fit twice (p = 8, 10), the
        // next stage's loads are issued before this stage is stored, so their latency overlaps
        constexpr int RPW = kBlkRows / kAblkLoadWarps / 32;  // rows per lane
        constexpr int CPR = CH / 8;                          // 16-byte chunks per row
        constexpr int NB = RPW * 2 * CPR;                    // chunks per lane and stage
        const int r0 = (kBlkRows / kAblkLoadWarps) * (warp - kLoad0) + lane;
        auto fetch = [&](int s, int4(&v)[NB]) {
            const int d = d_lo + s / NKC, c = s % NKC;
            const int kw = KD - c * CH < CH ? KD - c * CH : CH;
#pragma unroll
            for (int rr = 0; rr < RPW; ++rr) {
                const int64_t row = tsrc[d * kBlkRows + r0 + 32 * rr];
#pragma unroll
                for (int pl = 0; pl < 2; ++pl) {
                    const int4 *g = reinterpret_cast<const int4 *>(Apre + (row * 2 + pl) * KD + (int64_t)c * CH);
#pragma unroll
                    for (int q = 0; q < CPR; ++q) v[(rr * 2 + pl) * CPR + q] = 8 * q < kw ? __ldg(g + q) : int4{0, 0, 0, 0};
                }
            }
        };
        auto put = [&](int s, const int4(&v)[NB]) {
            const int st = s % NSTAGE, c = s % NKC;
            int ok = 1;
            if (s >= NSTAGE && lane == 0)
                ok = mbar_wait_bounded(&empty_bar[st], ((s / NSTAGE) - 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok || s_abort) {
                if (lane == 0) s_abort = 1;
                return false;
            }
            const int kw = KD - c * CH < CH ? KD - c * CH : CH;
#pragma unroll
            for (int rr = 0; rr < RPW; ++rr) {
                const int r = r0 + 32 * rr;
#pragma unroll
                for (int pl = 0; pl < 2; ++pl) {
                    unsigned char *dst = a_pl(st, pl) + (size_t)r * (2 * CH);
#pragma unroll
                    for (int q = 0; q < CPR; ++q) {
                        if (8 * q >= kw) break;
                        // the TMA's swizzle of this row: 16-byte chunk q at q ^ (row bits)
                        const int qs = CH == 64 ? (q ^ (r & 7)) : (q ^ ((r >> 1) & 3));
                        *reinterpret_cast<int4 *>(dst + 16 * qs) = v[(rr * 2 + pl) * CPR + q];
                    }
                }
            }
            fence_proxy_async();  // the generic-proxy stores, before the MMA's async-proxy reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[st]);
            return true;
        };
        if constexpr (NB <= 16) {
            int4 va[NB], vb[NB];
            if (S > 0) fetch(0, va);
            for (int s = 0; s < S; s += 2) {
                if (s + 1 < S) fetch(s + 1, vb);
                if (!put(s, va) || s + 1 >= S) break;
                if (s + 2 < S) fetch(s + 2, va);
                if (!put(s + 1, vb)) break;
            }
        } else {
            int4 va[NB];
            for (int s = 0; s < S; ++s) {
                fetch(s, va);
                if (!put(s, va)) break;
            }
        }
    } else if (warp == kProdWarp) {
        if (lane == 0) {
            for (int s = 0; s < S; ++s) {
                const int st = s % NSTAGE, d = d_lo + s / NKC, c = s % NKC;
                if (s >= NSTAGE &&
                    !mbar_wait_bounded(&empty_bar[st], ((s / NSTAGE) - 1) & 1, kWaitLimitNs, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                mbar_expect_tx(&full_bar[st], 2u * (uint32_t)C::B_BYTES);
                const int k0 = c * CH;
                blk_tma4(b_hi(st), &prm.tmB, k0, nt * C::NSTRIDE, 0, d, &full_bar[st]);
                blk_tma4(b_lo(st), &prm.tmB, k0, nt * C::NSTRIDE, 1, d, &full_bar[st]);
                s_issued[st] += 1;
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            for (int s = 0; s < S; ++s) {
                const int st = s % NSTAGE, c = s % NKC;
                const int uc = (c * DS) / NKC, u = (s / NKC) * DS + uc, b = u & 1;
                const bool first = c == 0 || ((c - 1) * DS) / NKC != uc;
                const bool last = c == NKC - 1 || ((c + 1) * DS) / NKC != uc;
                if (first && u >= 2 &&
                    !mbar_wait_bounded(&dempty[b], ((u - 2) >> 1) & 1, kWaitLimitNs, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                if (!mbar_wait_bounded(&full_bar[st], (s / NSTAGE) & 1, kWaitLimitNs, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const int kw = KD - c * CH < CH ? KD - c * CH : CH;
                const uint32_t ah = smem_u32(a_pl(st, 0)), al = smem_u32(a_pl(st, 1));
                const uint32_t bh = smem_u32(b_hi(st)), bl = smem_u32(b_lo(st));
                const uint32_t dt = tmem + (uint32_t)(b * NT);
                for (int j = 0; j < (kw + 15) / 16; ++j) {
                    const uint32_t o = 32u * j;
                    blk_mma_ss(dt, blk_desc<CH>(al + o), blk_desc<CH>(bh + o), kIdesc, (first && j == 0) ? 0u : 1u);
                    blk_mma_ss(dt, blk_desc<CH>(ah + o), blk_desc<CH>(bl + o), kIdesc, 1u);
                    blk_mma_ss(dt, blk_desc<CH>(ah + o), blk_desc<CH>(bh + o), kIdesc, 1u);
                }
                tc_commit(&empty_bar[st]);
                if (last) tc_commit(&dfull[b]);
            }
            tc_commit(&done_bar);
        }
    } else {
        // ===== drain warps: row r (target unit), columns [h NH, h NH + NH) of the N-tile =====
        const int quad = warp & 3, h = warp >> 2;
        const int r = 32 * quad + lane;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        const int64_t unit = ut * kBlkRows + r;
        const bool rok = unit < nu;
        const int g = *gexp;
        float acc[NH];
#pragma unroll
        for (int i = 0; i < NH; ++i) acc[i] = 0.f;
        bool alive = true;
        for (int u = 0; u < NU && alive; ++u) {
            const int d = d_lo + u / DS, b = u & 1;
            const int64_t row = tsrc[d * kBlkRows + r];
            const float f = row == prm.zrow ? 0.f : blk_pow2(-((int)uscale[row] + g));
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&dfull[b], (u >> 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                alive = false;
                break;
            }
            tc_fence_after();
            const uint32_t col0 = tmem + lane_base + (uint32_t)(b * NT + h * NH);
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += 32) {
                constexpr int W = 32;
                uint32_t v[W];
#pragma unroll
                for (int q = 0; q < W; q += 8)
                    if (c0 + q < NH) blk_ld8(col0 + (uint32_t)(c0 + q), v + q);
                tmem_wait_ld_regs(v);
#pragma unroll
                for (int q = 0; q < W; ++q)
                    if (c0 + q < NH) acc[c0 + q] = fmaf(__uint_as_float(v[q]), f, acc[c0 + q]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[b]);
        }
        if (!alive && lane == 0) s_abort = 1;
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&done_bar, 0u, kWaitLimitNs, nullptr) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) s_abort = 1;
        __syncwarp();
        if (ok && alive && !s_abort && rok) {
            float *dst = prm.ksplit > 1 ? Lpart + (int64_t)ks * prm.part_stride : Lc;
            const int64_t q = units[unit];
#pragma unroll
            for (int i = 0; i < NH; i += 4) {
                const int col = h * NH + i;
                const int gc = nt * C::NSTRIDE + col;
                if (col >= C::NSTRIDE || gc >= KD) continue;
                const int tau = gc / PP, n = gc % PP;
                const int32_t cell = child_of[q * 8 + tau];
                if (cell < 0) continue;
                *reinterpret_cast<float4 *>(dst + (int64_t)cell * PP + n) =
                    make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            atomicOr(status, kStatusTimeout);
            for (int st = 0; st < NSTAGE; ++st)
                if (s_issued[st] > 0) mbar_wait_bounded(&full_bar[st], (s_issued[st] - 1) & 1, kWaitLimitNs, nullptr);
        }
        __syncthreads();
    }
    if (warp == kMmaWarp) {
        __syncwarp();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// ---- sum of the offset ranges' partial sums (fixed order, so the result does not depend on
// which CTA finished first): Lc = sum_k Lpart[k] over the nonempty cells of levels 2..L
__global__ void __launch_bounds__(256) k_blk_reduce(int64_t c0, int64_t c1, int PP4, int ksplit, int64_t stride4,
                                                    const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
                                                    const float4 *__restrict__ part, float4 *__restrict__ Lc)
{
    const int64_t i = c0 * PP4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= c1 * PP4) return;
    const int64_t cell = i / PP4;
    if (end[cell] <= begin[cell]) return;
    float4 a = part[i];
    for (int k = 1; k < ksplit; ++k) {
        const float4 b = part[i + k * stride4];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    }
    Lc[i] = a;
}

// ---- host side ----------------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// per-level layout of the pre-split sources: parents of levels 1 .. L-1, level lp at parent
// offset level_offset(lp) - 1
int64_t blk_parents_before(int lp) { return level_offset(lp) - 1; }

}  // namespace

size_t m2l_blk_presplit_bytes(int P, int L)
{
    if (L < 2) return 0;
    return (size_t)blk_parents_before(L) * 2 * 8 * P * P * sizeof(__half);
}

size_t m2l_blk_scale_bytes(int L) { return L < 2 ? 0 : (size_t)blk_parents_before(L); }

// tiles of one launch over levels 2..L (ksplit 1)
template <int P>
static int blk_tiles(int L)
{
    int n = 0;
    for (int l = 2; l <= L; ++l) {
        const int pg = 1 << (l - 1);
        const int bx = pg < 8 ? pg : 8, by = pg < 4 ? pg : 4;
        n += (pg / bx) * (pg / by) * (pg / by) * BlkCfg<P, 64>::NTILES;
    }
    return n;
}

static int blk_tiles_p(int P, int L)
{
    switch (P) {
    case 4: return blk_tiles<4>(L);
    case 6: return blk_tiles<6>(L);
    case 8: return blk_tiles<8>(L);
    case 10: return blk_tiles<10>(L);
    }
    return 0;
}

// offset ranges per tile: 1 when there are at least kBlkFillCtas tiles (one per SM of a
// 152-SM GB300), else enough ranges for about twice that many CTAs (each range a whole number of
// offsets, at most 26).  A fixed rule, so that the workspace size does not depend on the device.
constexpr int kBlkFillCtas = 152;
int m2l_blk_ksplit(int P, int L)
{
    const int t = blk_tiles_p(P, L);
    if (L < 2 || t <= 0 || t >= kBlkFillCtas) return 1;
    const int k = (2 * kBlkFillCtas + t - 1) / t;
    return k < 26 ? k : 26;
}

// partial sums of the offset ranges: ksplit x (cells of levels 0..L) x p^2 floats (0 if not split)
size_t m2l_blk_part_bytes(int P, int L)
{
    const int k = m2l_blk_ksplit(P, L);
    return k > 1 ? (size_t)k * level_offset(L + 1) * P * P * sizeof(float) : 0;
}

size_t m2l_blk_table_bytes(int P)
{
    const size_t KD = 8 * (size_t)P * P;
    return 26 * 2 * KD * KD * sizeof(__half) + 256;
}

// the table: B (hi | lo per d) then, 256-aligned, the exponent g and the max-bits scratch word
void launch_build_m2l_blk(int P, const float *ops, void *table, cudaStream_t s)
{
    const size_t KD = 8 * (size_t)P * P;
    __half *B = static_cast<__half *>(table);
    int *g = reinterpret_cast<int *>(B + 26 * 2 * KD * KD);
    unsigned *mbits = reinterpret_cast<unsigned *>(g + 1);
    cudaMemsetAsync(mbits, 0, sizeof(unsigned), s);
    switch (P) {
    case 4:
        k_blk_opmax<4><<<kM2LCodes, 256, 0, s>>>(ops, mbits);
        k_blk_build<4><<<(unsigned)(26 * KD), 256, 0, s>>>(ops, mbits, B, g);
        break;
    case 6:
        k_blk_opmax<6><<<kM2LCodes, 256, 0, s>>>(ops, mbits);
        k_blk_build<6><<<(unsigned)(26 * KD), 256, 0, s>>>(ops, mbits, B, g);
        break;
    case 8:
        k_blk_opmax<8><<<kM2LCodes, 256, 0, s>>>(ops, mbits);
        k_blk_build<8><<<(unsigned)(26 * KD), 256, 0, s>>>(ops, mbits, B, g);
        break;
    case 10:
        k_blk_opmax<10><<<kM2LCodes, 256, 0, s>>>(ops, mbits);
        k_blk_build<10><<<(unsigned)(26 * KD), 256, 0, s>>>(ops, mbits, B, g);
        break;
    }
    note_launches(2);
}


void launch_blk_presplit(int P, int L, const int32_t *begin, const int32_t *end, const float *M, void *presplit,
                         int8_t *pscale, cudaStream_t s)
{
    const size_t KD = 8 * (size_t)P * P;
    for (int l = 2; l <= L; ++l) {
        const int64_t np = int64_t(1) << (3 * (l - 1));
        __half *A = static_cast<__half *>(presplit) + (size_t)blk_parents_before(l - 1) * 2 * KD;
        int8_t *sc = pscale + blk_parents_before(l - 1);
        const unsigned grid = (unsigned)((np + 7) / 8);
        switch (P) {
        case 4: k_blk_presplit<4><<<grid, 256, 0, s>>>(l, begin, end, M, A, sc); break;
        case 6: k_blk_presplit<6><<<grid, 256, 0, s>>>(l, begin, end, M, A, sc); break;
        case 8: k_blk_presplit<8><<<grid, 256, 0, s>>>(l, begin, end, M, A, sc); break;
        case 10: k_blk_presplit<10><<<grid, 256, 0, s>>>(l, begin, end, M, A, sc); break;
        }
        note_launches(1);
    }
}

template <int P, int CH>
static int launch_blk_t(int L, const int32_t *begin, const int32_t *end, const void *presplit,
                        const int8_t *pscale, const void *table, float *Lc, float *Lpart, int *status, cudaStream_t s,
                        int max_ctas)
{
    using C = BlkCfg<P, CH>;
    constexpr CUtensorMapSwizzle kSw = CH == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return -1;
    BlkParams prm;  // the kernel parameter (copied at launch)
    memset(&prm, 0, sizeof(prm));
    prm.L = L;
    const cuuint64_t KD = C::KD;
    const int *gexp = reinterpret_cast<const int *>(static_cast<const __half *>(table) + 26 * 2 * KD * KD);
    int ntiles = 0;
    for (int l = 2; l <= L; ++l) {
        const int pg = 1 << (l - 1);
        const int bx = pg < 8 ? pg : 8, by = pg < 4 ? pg : 4, bz = by;
        prm.tile_lo[l] = ntiles;
        ntiles += (pg / bx) * (pg / by) * (pg / bz) * C::NTILES;
        void *A = const_cast<__half *>(static_cast<const __half *>(presplit) + (size_t)blk_parents_before(l - 1) * 2 * KD);
        const cuuint64_t dims[5] = {KD, 2, (cuuint64_t)pg, (cuuint64_t)pg, (cuuint64_t)pg};
        const cuuint64_t strides[4] = {KD * 2, KD * 4, KD * 4 * pg, KD * 4 * pg * pg};
        const cuuint32_t box[5] = {(cuuint32_t)CH, 1, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&prm.tmA[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, A, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, kSw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    prm.tile_lo[L + 1] = ntiles;
    prm.ksplit = m2l_blk_ksplit(P, L);
    prm.part_stride = level_offset(L + 1) * C::PP;
    if (prm.ksplit > 1 && !Lpart) return -1;
    {
        const cuuint64_t dims[4] = {KD, KD, 2, 26};
        const cuuint64_t strides[3] = {KD * 2, KD * KD * 2, KD * KD * 4};
        const cuuint32_t box[4] = {(cuuint32_t)CH, (cuuint32_t)C::NT, 1, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&prm.tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(table), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, kSw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    auto kern = k_m2l_blk<P, kBlkDrainsPerOffset, CH>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmemBytes);
    const int nctas = ntiles * prm.ksplit;
    const int step = max_ctas > 0 ? max_ctas : nctas;
    for (int t0 = 0; t0 < nctas; t0 += step) {
        prm.tile0 = t0;
        const int gsz = nctas - t0 < step ? nctas - t0 : step;
        kern<<<gsz, kBlkThreads, C::kSmemBytes, s>>>(prm, begin, end, pscale, gexp, Lc, Lpart, status);
        note_launches(1);
    }
    if (prm.ksplit > 1) {
        const int64_t c0 = level_offset(2), c1 = level_offset(L + 1), PP4 = C::PP / 4;
        const int64_t nthr = (c1 - c0) * PP4;
        k_blk_reduce<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(
            c0, c1, (int)PP4, prm.ksplit, prm.part_stride / 4, begin, end, reinterpret_cast<const float4 *>(Lpart),
            reinterpret_cast<float4 *>(Lc));
        note_launches(1);
    }
    return 0;
}

// M2L of levels 2..L of the uniform tree (table: launch_build_m2l_blk; presplit/pscale:
// launch_blk_presplit after the upward pass); -1 if the tensor maps cannot be encoded
int launch_m2l_blk(int P, int L, const int32_t *begin, const int32_t *end, const void *presplit,
                   const int8_t *pscale, const void *table, float *Lc, float *Lpart, int *status, cudaStream_t s,
                   int max_ctas)
{
    if (L < 2) return 0;
    // p = 8, 10: four stages of 32-wide K chunks (64-byte swizzle) cover the TMA latency better
    // than two of 64 (1M, p = 10: 0.343 against 0.372 ms); p = 4, 6 fit three 64-wide stages
    switch (P) {
    case 4: return launch_blk_t<4, 64>(L, begin, end, presplit, pscale, table, Lc, Lpart, status, s, max_ctas);
    case 6: return launch_blk_t<6, 64>(L, begin, end, presplit, pscale, table, Lc, Lpart, status, s, max_ctas);
    case 8: return launch_blk_t<8, 32>(L, begin, end, presplit, pscale, table, Lc, Lpart, status, s, max_ctas);
    case 10: return launch_blk_t<10, 32>(L, begin, end, presplit, pscale, table, Lc, Lpart, status, s, max_ctas);
    }
    return -1;
}

// ---- adaptive tree ----------------------------------------------------------------------------
size_t m2l_ablk_presplit_bytes(int P, int64_t ucap) { return (size_t)(ucap + 1) * 2 * 8 * P * P * sizeof(__half); }

int64_t m2l_ablk_tiles_units(int64_t ucap) { return (ucap + kBlkRows - 1) / kBlkRows * kBlkRows; }

size_t m2l_ablk_src_bytes(int64_t ucap) { return (size_t)m2l_ablk_tiles_units(ucap) * 26 * sizeof(int32_t); }

// offset ranges per tile from the particle count and leaf size alone (an estimate of the units:
// a quarter of n / leaf_size), so that evaluations of the same count split alike whatever their
// trees (a captured batch and the same instance alone sum in the same order)
int m2l_ablk_ksplit(int P, int64_t n, int leaf_size)
{
    const int nt = P == 4 ? BlkCfg<4, 64>::NTILES : P == 6 ? BlkCfg<6, 64>::NTILES : P == 8 ? BlkCfg<8, 32>::NTILES
                                                                                            : BlkCfg<10, 32>::NTILES;
    const int64_t units = n / (4 * (int64_t)(leaf_size > 0 ? leaf_size : 1)) + 1;
    const int64_t t = (units + kBlkRows - 1) / kBlkRows * nt;
    if (t <= 0 || t >= kBlkFillCtas) return 1;
    const int64_t k = (2 * kBlkFillCtas + t - 1) / t;
    return k < 26 ? (int)k : 26;
}

void launch_ablk_prep(int P, Span cells, int64_t ucap, const int32_t *level, const int32_t *nchild,
                      const int32_t *child_of, const int32_t *coll, const float *M, uint32_t *flag, uint32_t *scan,
                      uint32_t *scan_tmp, int32_t *unit_of, int32_t *units, int32_t *n_units, void *Apre,
                      int8_t *uscale, int32_t *src, cudaStream_t s)
{
    const unsigned gc = (unsigned)((cells.cap + 255) / 256);
    k_ablk_flags<<<gc, 256, 0, s>>>(cells, level, nchild, flag);
    launch_exclusive_scan(flag, scan, cells.cap, scan_tmp, s);
    k_ablk_units<<<gc, 256, 0, s>>>(cells, flag, scan, unit_of, units, n_units);
    const int64_t zrow = ucap;
    const unsigned gp = (unsigned)((ucap + 1 + 7) / 8);
    __half *A = static_cast<__half *>(Apre);
    switch (P) {
    case 4: k_ablk_presplit<4><<<gp, 256, 0, s>>>(n_units, zrow, units, child_of, M, A, uscale); break;
    case 6: k_ablk_presplit<6><<<gp, 256, 0, s>>>(n_units, zrow, units, child_of, M, A, uscale); break;
    case 8: k_ablk_presplit<8><<<gp, 256, 0, s>>>(n_units, zrow, units, child_of, M, A, uscale); break;
    case 10: k_ablk_presplit<10><<<gp, 256, 0, s>>>(n_units, zrow, units, child_of, M, A, uscale); break;
    }
    const int64_t up = m2l_ablk_tiles_units(ucap);
    k_ablk_src<<<(unsigned)((up * 26 + 255) / 256), 256, 0, s>>>(n_units, up, zrow, units, coll, unit_of, src);
    note_launches(4);
}

template <int P, int CH>
static int launch_ablk_t(int64_t ucap, const int32_t *n_units, const int32_t *units, const int32_t *child_of,
                         const int32_t *src, const void *Apre, const int8_t *uscale, const void *table, float *Lc,
                         float *Lpart, int ksplit, int64_t part_stride, int *status, cudaStream_t s, int max_ctas)
{
    using C = BlkCfg<P, CH>;
    constexpr CUtensorMapSwizzle kSw = CH == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return -1;
    AblkParams prm;
    memset(&prm, 0, sizeof(prm));
    const cuuint64_t KD = C::KD;
    const int *gexp = reinterpret_cast<const int *>(static_cast<const __half *>(table) + 26 * 2 * KD * KD);
    {
        const cuuint64_t dims[4] = {KD, KD, 2, 26};
        const cuuint64_t strides[3] = {KD * 2, KD * KD * 2, KD * KD * 4};
        const cuuint32_t box[4] = {(cuuint32_t)CH, (cuuint32_t)C::NT, 1, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&prm.tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(table), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, kSw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    prm.ksplit = ksplit;
    prm.part_stride = part_stride;
    prm.zrow = ucap;
    if (ksplit > 1 && !Lpart) return -1;
    auto kern = k_m2l_ablk<P, kBlkDrainsPerOffset, CH>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmemBytes);
    const int64_t nctas64 = (ucap + kBlkRows - 1) / kBlkRows * C::NTILES * ksplit;
    const int nctas = (int)nctas64;
    const int step = max_ctas > 0 ? max_ctas : nctas;
    for (int t0 = 0; t0 < nctas; t0 += step) {
        prm.tile0 = t0;
        const int gsz = nctas - t0 < step ? nctas - t0 : step;
        kern<<<gsz, kAblkThreads, C::kSmemBytes, s>>>(prm, n_units, units, child_of, src,
                                                      static_cast<const __half *>(Apre), uscale, gexp, Lc, Lpart,
                                                      status);
        note_launches(1);
    }
    return 0;
}

int launch_m2l_ablk(int P, int64_t ucap, const int32_t *n_units, const int32_t *units, const int32_t *child_of,
                    const int32_t *src, const void *Apre, const int8_t *uscale, const void *table, float *Lc,
                    float *Lpart, int ksplit, int64_t part_stride, int *status, cudaStream_t s, int max_ctas)
{
    if (ucap <= 0) return 0;
    switch (P) {
    case 4: return launch_ablk_t<4, 64>(ucap, n_units, units, child_of, src, Apre, uscale, table, Lc, Lpart, ksplit, part_stride, status, s, max_ctas);
    case 6: return launch_ablk_t<6, 64>(ucap, n_units, units, child_of, src, Apre, uscale, table, Lc, Lpart, ksplit, part_stride, status, s, max_ctas);
    case 8: return launch_ablk_t<8, 32>(ucap, n_units, units, child_of, src, Apre, uscale, table, Lc, Lpart, ksplit, part_stride, status, s, max_ctas);
    case 10: return launch_ablk_t<10, 32>(ucap, n_units, units, child_of, src, Apre, uscale, table, Lc, Lpart, ksplit, part_stride, status, s, max_ctas);
    }
    return -1;
}

// Lc = the sum of the offset ranges' partial sums, in range order, over the cells of `deep`
__global__ void __launch_bounds__(256) k_ablk_reduce(Span deep, int PP4, int ksplit, int64_t stride4,
                                                     const float4 *__restrict__ part, float4 *__restrict__ Lc)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= span_count(deep) * PP4) return;
    const int64_t i = span_first(deep) * PP4 + j;
    float4 a = part[i];
    for (int k = 1; k < ksplit; ++k) {
        const float4 b = part[i + k * stride4];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    }
    Lc[i] = a;
}

void launch_ablk_reduce(int P, Span deep, int ksplit, int64_t part_stride, const float *Lpart, float *Lc,
                        cudaStream_t s)
{
    const int64_t PP4 = (int64_t)P * P / 4;
    const int64_t nthr = deep.cap * PP4;
    if (nthr <= 0) return;
    k_ablk_reduce<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(deep, (int)PP4, ksplit, part_stride / 4,
                                                                 reinterpret_cast<const float4 *>(Lpart),
                                                                 reinterpret_cast<float4 *>(Lc));
    note_launches(1);
}

}  // namespace gbfmm
