// M2L (Eq. 4) on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// The contraction is the one of the CUDA-core kernel: for a tile of targets of one level and
// one child position tau, and each of the 189 admissible offsets o (ascending stencil code),
//     L~(t, :) += T_o M~(src(t, o), :)          (real-packed, side-scaled expansions).
// Here the 128 targets of a tile are the MMA's M dimension (one TMEM lane per target), the
// p^2 output rows of T_o its N dimension (padded to a multiple of 16) and the p^2 input
// coefficients its K dimension (padded to a multiple of 8):
//     D[128 x N] (TMEM, FP32) += A[128 x K] (gathered source expansions) * B[N x K]^T (T_o).
// FP32 accuracy from TF32 operands (3xTF32): every operand is split x = hi + lo with hi rounded
// to TF32, and D accumulates hi*hi + lo*hi + hi*lo; the dropped lo*lo term and the TF32
// rounding (operator table) or truncation (sources, in the tensor core) of lo are below 2^-21
// of |x|.  The operator halves are split once, when the table is built; the source halves by
// the threads that gather them.
//
// Pipeline (one CTA per tile, warp-specialised, NSTAGE stages; a stage is one K-chunk of one
// offset).  The A operand lives in tensor memory, so shared memory carries only the operator:
//   warps 0-7, converters (two per TMEM lane quadrant; thread = target row, K half h): walk the
//     target's CSR list, load each step's source K-chunk into registers two steps ahead (zeros
//     for a missing source or k >= p^2), split it into TF32 halves and store them with
//     tcgen05.st into the stage's A_hi / A_lo columns of its TMEM lane; warp 0 also starts the
//     bulk copies of the operator chunk (B_hi | B_lo, stored pre-laid-out in the canonical
//     no-swizzle K-major layout in global memory) on the stage's "full" mbarrier;
//   warp 8: allocates TMEM; one thread waits on "full", issues the MMAs of the stage (3 per
//     8-wide K step, A from TMEM, B from shared memory) and commits them to "empty";
//   drains (warps 0-7): offset o accumulates into TMEM accumulator o & 1 (a chain of 3 x K/8
//     MMAs).  Once it is complete, each thread loads half of its TMEM lane (its target's row of
//     the partial) and adds it to FP32 registers, then releases the accumulator for offset
//     o + 2.  The tensor cores' accumulation rounds toward zero; short chains keep that bias at
//     a few units of 2^-24, and the sum over the 189 offsets is rounded to nearest;
//   epilogue: each thread writes its half of its target's p^2 local coefficients.
// Every wait is bounded (1 s of %globaltimer); on timeout the kernel raises the status word,
// lets its copies and MMAs in flight finish (bounded), frees its TMEM and returns.
#include "common.cuh"
#include "ptx.cuh"

#include <stdlib.h>

namespace gbfmm {

__constant__ uint16_t c_tc_codes[8][189];

void init_m2l_tc_constants()
{
    uint16_t codes[8][189];
    for (int t = 0; t < 8; ++t) {
        int cx = t & 1, cy = (t >> 1) & 1, cz = (t >> 2) & 1, k = 0;
        for (int oz = -2 - cz; oz <= 3 - cz; ++oz)
            for (int oy = -2 - cy; oy <= 3 - cy; ++oy)
                for (int ox = -2 - cx; ox <= 3 - cx; ++ox) {
                    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                    codes[t][k++] = (uint16_t)m2l_code(ox, oy, oz);
                }
    }
    cudaMemcpyToSymbol(c_tc_codes, codes, sizeof(codes));
}

// Shapes per order.  KS = K steps of 8 per offset, split into NCH chunks of (nearly) equal size
// (at most CK steps each); NS pipeline stages; Q converter warps per TMEM lane quadrant.
template <int P, int CK, int NS, int Q = 2>
struct TcCfg {
    static constexpr int PP = P * P;
    static constexpr int KP = (PP + 7) / 8 * 8;      // K, padded to the MMA's K step
    static constexpr int NP = (PP + 15) / 16 * 16;   // N, padded to a multiple of 16
    static constexpr int NH = NP / Q;                // output columns drained per thread
    static constexpr int KS = KP / 8;
    static constexpr int NCH = (KS + CK - 1) / CK;
    static constexpr int KCMAX = 8 * ((KS + NCH - 1) / NCH);  // K width of the largest chunk
    static constexpr int TM = 128;                   // targets per tile (MMA M)
    static constexpr int NSTAGE = NS;
    // TMEM: two accumulators D0, D1 (NP columns each) at column 0, A stages (A_hi | A_lo, 32
    // columns each) from column 256
    static constexpr int TMEM_COLS = 512;
    static constexpr int A_COL0 = 256;
    static constexpr int B_FLOATS = 2 * NP * KCMAX;  // one stage: B_hi | B_lo
    // at least 116 KB of shared memory: one CTA per SM, so the whole of TMEM is this CTA's
    static constexpr size_t kStageBytes = (size_t)NSTAGE * B_FLOATS * sizeof(float);
    static constexpr size_t kSmemBytes = kStageBytes > 116 * 1024 ? kStageBytes : 116 * 1024;
    static constexpr int NCONV = 4 * Q;              // converter warps (Q per TMEM lane quadrant)
    static constexpr int NF = KCMAX / 4 / Q;         // float4 columns of a chunk per converter thread
    static constexpr int NTHREADS = 32 * NCONV + 32; // + one MMA warp
    static_assert((KCMAX / 4) % Q == 0 && NH % 4 == 0, "converter split");
    static_assert(NP >= 16 && NP <= 128 && NP % 16 == 0, "MMA N (two accumulators below column 256)");
    static_assert(KCMAX <= 32, "a K chunk fits a 32-column TMEM slot");
    static_assert(A_COL0 + 64 * NS <= TMEM_COLS, "TMEM A stages");
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};

// operator table per offset code: T_hi then T_lo, each [KP/4][NP][4] (the canonical no-swizzle
// K-major layout of the N x K operand; a K-chunk [k0, k0 + kw) is the contiguous range
// starting at float k0 * NP)
template <int P>
struct TcTable {
    static constexpr int PP = P * P, PR = (PP + 7) / 8 * 8, KP = (PP + 7) / 8 * 8, NP = (PP + 15) / 16 * 16;
    static constexpr int HALF = KP * NP;
    static constexpr int CODE_FLOATS = 2 * HALF;
};

GB_DEV void chunk_range(int c, int KS, int NCH, int &k0, int &kw)
{
    const int s0 = (c * KS) / NCH, s1 = ((c + 1) * KS) / NCH;
    k0 = 8 * s0;
    kw = 8 * (s1 - s0);
}

size_t m2l_tc_table_floats(int P)
{
    switch (P) {
    case 4: return (size_t)kM2LCodes * TcTable<4>::CODE_FLOATS;
    case 6: return (size_t)kM2LCodes * TcTable<6>::CODE_FLOATS;
    case 8: return (size_t)kM2LCodes * TcTable<8>::CODE_FLOATS;
    case 10: return (size_t)kM2LCodes * TcTable<10>::CODE_FLOATS;
    }
    return 0;
}

// rows n >= p^2 and columns k >= p^2 zero
template <int P>
__global__ void k_build_m2l_tc(const float *__restrict__ ops, float *__restrict__ tc)
{
    using T = TcTable<P>;
    const int code = blockIdx.x;
    float *blk = tc + (size_t)code * T::CODE_FLOATS;
    for (int e = threadIdx.x; e < T::NP * T::KP; e += blockDim.x) {
        const int n = e / T::KP, k = e % T::KP;
        const float v = (n < T::PP && k < T::PP) ? ops[((size_t)code * T::PP + k) * T::PR + n] : 0.f;
        const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
        const int o = (k >> 2) * T::NP * 4 + n * 4 + (k & 3);
        blk[o] = hi;
        blk[T::HALF + o] = lo;
    }
}

void launch_build_m2l_tc(int P, const float *ops, float *tc, cudaStream_t s)
{
    switch (P) {
    case 4: k_build_m2l_tc<4><<<kM2LCodes, 256, 0, s>>>(ops, tc); break;
    case 6: k_build_m2l_tc<6><<<kM2LCodes, 256, 0, s>>>(ops, tc); break;
    case 8: k_build_m2l_tc<8><<<kM2LCodes, 256, 0, s>>>(ops, tc); break;
    case 10: k_build_m2l_tc<10><<<kM2LCodes, 256, 0, s>>>(ops, tc); break;
    }
    note_launches(1);
}

struct TcTiles {
    int L;
    int ntiles_level[kMaxLevel + 1];
};

template <int P, int CK, int NS, int GRP, int Q>
__global__ void __launch_bounds__(TcCfg<P, CK, NS, Q>::NTHREADS, 1)
    k_m2l_tc(TcTiles tiles, const int4 *__restrict__ tdesc, const int32_t *__restrict__ tlist,
             const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
             const uint32_t *__restrict__ m2l_offs, const int32_t *__restrict__ m2l_ids,
             const uint16_t *__restrict__ m2l_code, const float *__restrict__ optc, const float *__restrict__ M,
             float *__restrict__ Lc, int *status)
{
    using C = TcCfg<P, CK, NS, Q>;
    using T = TcTable<P>;
    constexpr int PP = C::PP, NP = C::NP, NH = C::NH, TM = C::TM, NSTAGE = C::NSTAGE, NCH = C::NCH, NF = C::NF;
    constexpr int S = 189 * NCH;
    constexpr int NGRP = (189 + GRP - 1) / GRP;  // accumulation chains (GRP offsets each)
    constexpr uint32_t kIdesc = tc_idesc_tf32(TM, NP);
    constexpr int kMmaWarp = C::NCONV;

    extern __shared__ __align__(1024) float tsm[];
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], drain_full[2], drain_empty[2], done_bar;
    __shared__ int s_issued[NSTAGE];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    // ---- tile: dense uniform levels (descending), or an explicit list (level, tau, start, count)
    int tau;
    int64_t q0 = 0, nq = 0, off = 0, tstart = 0;
    int tcount = 0;
    if (tdesc) {
        const int4 d = tdesc[blockIdx.x];
        tau = d.y;
        tstart = d.z;
        tcount = d.w;
    } else {
        int rem = blockIdx.x;
        int l = tiles.L;
        while (l >= 2 && rem >= tiles.ntiles_level[l]) {
            rem -= tiles.ntiles_level[l];
            --l;
        }
        if (l < 2) return;
        nq = int64_t(1) << (3 * (l - 1));
        const int64_t qtiles = (nq + TM - 1) / TM;
        tau = (int)(rem / qtiles);
        q0 = (rem % qtiles) * TM;
        off = level_offset(l);
    }
    auto target = [&](int t) -> int64_t {
        if (tdesc) return t < tcount ? (int64_t)tlist[tstart + t] : -1;
        const int64_t q = q0 + t;
        return q < nq ? off + 8 * q + tau : -1;
    };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < NSTAGE; ++st) {
            mbar_init(&full_bar[st], C::NCONV + 1);  // converter warps + the operator copies' expect_tx
            mbar_init(&empty_bar[st], 1);  // one tcgen05.commit
            s_issued[st] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&drain_full[b], 1);   // tcgen05.commit after an offset's last MMA
            mbar_init(&drain_empty[b], C::NCONV);  // the draining (converter) warps
        }
        mbar_init(&done_bar, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) tmem_alloc(&s_tmem, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < kMmaWarp) {
        // ====== converters / drainers: target row r; float4 columns [h NF, h NF + NF) of each
        // chunk; output columns [h NH, h NH + NH) ======
        const int quad = warp & 3, h = warp >> 2;
        const int r = 32 * quad + lane;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        const int64_t g = target(r);
        uint32_t ptr = 0, pend = 0;
        if (g >= 0 && end[g] > begin[g]) {
            ptr = m2l_offs[g];
            pend = m2l_offs[g + 1];
        }
        // the target's next list entry (code, source), read one entry ahead so that its latency
        // is hidden behind the offsets before it
        int nxt_code = 0xffff, nxt_id = 0;
        if (ptr < pend) {
            nxt_code = m2l_code[ptr];
            nxt_id = m2l_ids[ptr];
        }
        // source chunks are loaded into registers two steps ahead of their conversion
        const float *lsrc = nullptr;
        auto load = [&](int s2, float4 (&buf)[NF]) {
#pragma unroll
            for (int i = 0; i < NF; ++i) buf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (s2 >= S) return;
            const int oc2 = s2 / NCH, c2 = s2 % NCH;
            int k0, kw;
            chunk_range(c2, C::KS, NCH, k0, kw);
            if (c2 == 0) {
                lsrc = nullptr;
                if (nxt_code == (int)c_tc_codes[tau][oc2]) {
                    lsrc = M + (size_t)nxt_id * PP;
                    ++ptr;
                    nxt_code = 0xffff;
                    if (ptr < pend) {
                        nxt_code = m2l_code[ptr];
                        nxt_id = m2l_ids[ptr];
                    }
                }
            }
            if (!lsrc) return;
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                const int kk = 4 * (h * NF + i), k = k0 + kk;
                if (kk < kw && k < PP) buf[i] = __ldg(reinterpret_cast<const float4 *>(lsrc + k));
            }
        };
        // FP32 sum over offsets of the per-offset TMEM partials (each a chain of few MMAs)
        float acc[NH];
#pragma unroll
        for (int n = 0; n < NH; ++n) acc[n] = 0.f;
        auto drain = [&](int gi) -> bool {
            const int b = gi & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&drain_full[b], (gi >> 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) return false;
            tc_fence_after();
            constexpr int W = NH % 8 == 0 ? 8 : 4;
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += W) {
                uint32_t v[W];
                tmem_ld_cols(tmem + lane_base + (uint32_t)(b * NP + h * NH + c0), v);
#pragma unroll
                for (int j = 0; j < W; ++j) acc[c0 + j] += __uint_as_float(v[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drain_empty[b]);
            return true;
        };
        bool alive = true;
        auto step = [&](int s, float4 (&cur)[NF]) {
            const int st = s % NSTAGE, oc = s / NCH, c = s % NCH;
            if (s >= NSTAGE) {
                int ok = 1;
                if (lane == 0)
                    ok = mbar_wait_bounded(&empty_bar[st], ((s / NSTAGE) - 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    alive = false;
                    return;
                }
            }
            int k0, kw;
            chunk_range(c, C::KS, NCH, k0, kw);
            if (warp == 0 && lane == 0) {
                const int code = c_tc_codes[tau][oc];
                const uint32_t half = (uint32_t)NP * kw * 4u;
                const float *tb = optc + (size_t)code * T::CODE_FLOATS + (size_t)k0 * NP;
                float *B = tsm + (size_t)st * C::B_FLOATS;
                mbar_expect_tx(&full_bar[st], 2u * half);
                tma_bulk_g2s(B, tb, half, &full_bar[st]);
                tma_bulk_g2s(B + NP * kw, tb + T::HALF, half, &full_bar[st]);
                s_issued[st] += 1;
            }
            // split into TF32 halves and store the thread's 16 columns of A_hi and A_lo (its
            // TMEM lane = its target row)
            // hi = x rounded to TF32 (nearest, ties away: add half a TF32 unit to the magnitude's
            // bits and clear the 13 low bits); lo = x - hi exactly, which the tensor core reads
            // truncated to TF32 (error < 2^-21 |x|)
            const uint32_t acol = (uint32_t)(C::A_COL0 + 64 * st + 4 * h * NF);
            uint32_t hi[4 * NF], lo[4 * NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                const float x[4] = {cur[i].x, cur[i].y, cur[i].z, cur[i].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t hb = (__float_as_uint(x[e]) + 0x1000u) & 0xFFFFE000u;
                    hi[4 * i + e] = hb;
                    lo[4 * i + e] = __float_as_uint(x[e] - __uint_as_float(hb));
                }
            }
            tmem_st_cols(tmem + lane_base + acol, hi);
            tmem_st_cols(tmem + lane_base + acol + 32, lo);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[st]);
            load(s + 2, cur);
            // the previous chain's partial is complete once the next chain's first offset is queued
            if (c == NCH - 1 && oc >= 1 && (oc - 1) % GRP == GRP - 1 && !drain((oc - 1) / GRP)) alive = false;
        };
        float4 b0[NF], b1[NF];
        load(0, b0);
        load(1, b1);
        for (int s = 0; s < S && alive; s += 2) {
            step(s, b0);
            if (s + 1 < S && alive) step(s + 1, b1);
        }
        if (alive && !drain(NGRP - 1)) alive = false;
        if (!alive && lane == 0) s_abort = 1;
        // every MMA has completed once done_bar has (bounded; needed before TMEM is freed)
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&done_bar, 0u, kWaitLimitNs, nullptr) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) s_abort = 1;
        __syncwarp();
        if (ok && alive && !s_abort && g >= 0 && end[g] > begin[g]) {
#pragma unroll
            for (int n = 0; n < NH; n += 4)
                if (h * NH + n < PP)
                    *reinterpret_cast<float4 *>(Lc + g * PP + h * NH + n) =
                        make_float4(acc[n], acc[n + 1], acc[n + 2], acc[n + 3]);
        }
    } else if (lane == 0) {
        // ======= MMA issuer: chain gi (offsets GRP gi .. GRP gi + GRP - 1) accumulates in TMEM buffer gi & 1 =======
        for (int s = 0; s < S; ++s) {
            const int st = s % NSTAGE, oc = s / NCH, c = s % NCH, gi = oc / GRP, b = gi & 1;
            const bool chain_start = c == 0 && oc % GRP == 0;
            if (chain_start && gi >= 2 &&
                !mbar_wait_bounded(&drain_empty[b], ((gi - 2) >> 1) & 1, kWaitLimitNs, &s_abort)) {
                s_abort = 1;
                break;
            }
            if (!mbar_wait_bounded(&full_bar[st], (s / NSTAGE) & 1, kWaitLimitNs, &s_abort)) {
                s_abort = 1;
                break;
            }
            tc_fence_after();
            int k0, kw;
            chunk_range(c, C::KS, NCH, k0, kw);
            const float *Bhi = tsm + (size_t)st * C::B_FLOATS, *Blo = Bhi + NP * kw;
            const uint32_t d = tmem + (uint32_t)(b * NP);
            const uint32_t ahi = tmem + (uint32_t)(C::A_COL0 + 64 * st), alo = ahi + 32;
            for (int j = 0; j < kw / 8; ++j) {
                const uint64_t bh = smem_desc(Bhi + j * 2 * NP * 4, NP * 16, 128);
                const uint64_t bl = smem_desc(Blo + j * 2 * NP * 4, NP * 16, 128);
                // the small cross terms first, the hi*hi term last
                tc_mma_tf32_ta(d, alo + 8 * j, bh, kIdesc, (chain_start && j == 0) ? 0u : 1u);
                tc_mma_tf32_ta(d, ahi + 8 * j, bl, kIdesc, 1u);
                tc_mma_tf32_ta(d, ahi + 8 * j, bh, kIdesc, 1u);
            }
            tc_commit(&empty_bar[st]);
            if (c == NCH - 1 && (oc % GRP == GRP - 1 || oc == 188)) tc_commit(&drain_full[b]);
        }
        tc_commit(&done_bar);  // completes once every MMA issued above has completed
    }

    tc_fence_before();
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            atomicOr(status, kStatusTimeout);
            // let every issued operator copy land before the shared memory is released (bounded)
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

template <int P, int CK, int NS, int GRP = 1, int Q = 2>
static void launch_m2l_tc_t(const TcTiles &tiles, int grid, const int4 *tdesc, const int32_t *tlist,
                            const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                            const int32_t *m2l_ids, const uint16_t *m2l_code, const float *optc, const float *M,
                            float *Lc, int *status, cudaStream_t s)
{
    using C = TcCfg<P, CK, NS, Q>;
    cudaFuncSetAttribute(k_m2l_tc<P, CK, NS, GRP, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)C::kSmemBytes);
    k_m2l_tc<P, CK, NS, GRP, Q><<<grid, C::NTHREADS, C::kSmemBytes, s>>>(tiles, tdesc, tlist, begin, end, m2l_offs,
                                                                  m2l_ids, m2l_code, optc, M, Lc, status);
    note_launches(1);
}

// pipeline shape (GBFMM_M2L_TC_CFG, p = 10): 0 = chunks of <= 4 K steps, 4 stages; 1 = 4 steps,
// 2 stages; 2 = 2 steps, 4 stages; 3 = 3 steps, 4 stages; 4, 5 = as 0 with 2, 3 offsets per
// TMEM accumulation chain; 6, 7 = as 0 with 4, 1 converter warps per TMEM lane quadrant
static int tc_variant()
{
    static const int v = [] {
        const char *e = getenv("GBFMM_M2L_TC_CFG");
        const int x = e ? atoi(e) : 0;
        return (x >= 0 && x <= 7) ? x : 0;
    }();
    return v;
}

static void dispatch_tc(int P, const TcTiles &tiles, int grid, const int4 *tdesc, const int32_t *tlist,
                        const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                        const uint16_t *m2l_code, const float *optc, const float *M, float *Lc, int *status,
                        cudaStream_t s)
{
#define GBFMM_TC_ARGS tiles, grid, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s
    switch (P) {
    case 4: launch_m2l_tc_t<4, 2, 4>(GBFMM_TC_ARGS); break;
    case 6: launch_m2l_tc_t<6, 4, 4>(GBFMM_TC_ARGS); break;
    case 8: launch_m2l_tc_t<8, 4, 4>(GBFMM_TC_ARGS); break;
    case 10:
        switch (tc_variant()) {
        case 1: launch_m2l_tc_t<10, 4, 2>(GBFMM_TC_ARGS); break;
        case 2: launch_m2l_tc_t<10, 2, 4>(GBFMM_TC_ARGS); break;
        case 3: launch_m2l_tc_t<10, 3, 4>(GBFMM_TC_ARGS); break;
        case 4: launch_m2l_tc_t<10, 4, 4, 2>(GBFMM_TC_ARGS); break;
        case 5: launch_m2l_tc_t<10, 4, 4, 3>(GBFMM_TC_ARGS); break;
        case 6: launch_m2l_tc_t<10, 4, 4, 1, 4>(GBFMM_TC_ARGS); break;
        case 7: launch_m2l_tc_t<10, 4, 4, 1, 1>(GBFMM_TC_ARGS); break;
        default: launch_m2l_tc_t<10, 4, 4>(GBFMM_TC_ARGS); break;
        }
        break;
    }
#undef GBFMM_TC_ARGS
}

void launch_m2l_tc(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                   const int32_t *m2l_ids, const uint16_t *m2l_code, const float *optc, const float *M, float *Lc,
                   int *status, cudaStream_t s)
{
    if (L < 2) return;
    TcTiles tiles{};
    tiles.L = L;
    int total = 0;
    for (int l = 2; l <= L; ++l) {
        const int64_t nq = int64_t(1) << (3 * (l - 1));
        tiles.ntiles_level[l] = (int)(8 * ((nq + kM2LTcTargetsPerTile - 1) / kM2LTcTargetsPerTile));
        total += tiles.ntiles_level[l];
    }
    if (total == 0) return;
    dispatch_tc(P, tiles, total, nullptr, nullptr, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s);
}

void launch_m2l_tc_tiles(int P, const int4 *tdesc, int ntiles, const int32_t *tlist, const int32_t *begin,
                         const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                         const uint16_t *m2l_code, const float *optc, const float *M, float *Lc, int *status,
                         cudaStream_t s)
{
    if (ntiles <= 0) return;
    TcTiles tiles{};
    dispatch_tc(P, tiles, ntiles, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s);
}

int m2l_tc_mode()
{
    static const int mode = [] {
        const char *e = getenv("GBFMM_M2L_TC");
        const int v = e ? atoi(e) : 2;
        return (v == 0 || v == 1 || v == 2 || v == 4) ? v : 2;
    }();
    return mode;
}

bool m2l_use_tc() { return m2l_tc_mode() != 0; }

}  // namespace gbfmm
