// M2L (Eq. 4) on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// The contraction is the one of the CUDA-core kernel: for a tile of targets of one level and
// one child position tau, and each of the 189 admissible offsets o (ascending stencil code),
//     L~(t, :) += T_o M~(src(t, o), :)          (real-packed, side-scaled expansions).
// Here the 128 targets of a tile are the MMA's M dimension (one TMEM lane per target), the
// p^2 output rows of T_o its N dimension (padded to a multiple of 16) and the p^2 input
// coefficients its K dimension (padded to a multiple of 8):
//     D[128 x N] (TMEM, FP32) += A[128 x K] (gathered source expansions) * B[N x K]^T (T_o).
// FP32 accuracy from TF32 operands (3xTF32): every operand is split x = hi + lo with hi and lo
// rounded to TF32, and D accumulates hi*hi + lo*hi + hi*lo; the dropped lo*lo term and the
// rounding of lo are below 2^-21 of |x|.  The operator halves are split once, when the table
// is built; the source halves are split by the threads that gather them.
//
// Pipeline (one CTA per tile, warp-specialised, NSTAGE shared-memory stages; a stage holds
// one K-chunk of one offset):
//   warps 0-3 (one thread per target): walk the target's CSR list, load the source's K-chunk
//     (float4, zeros for a missing source), split it and store A_hi / A_lo in the canonical
//     no-swizzle K-major layout; warp 0 also starts the bulk copy of the operator chunk
//     (B_hi | B_lo, stored pre-laid-out in global memory) on the stage's "full" mbarrier;
//   warp 4: allocates the TMEM accumulator; one thread waits on "full", issues the MMAs of
//     the stage (3 per 8-wide K step) and commits them to the stage's "empty" mbarrier;
//   drains (warps 0-3): offset o accumulates into TMEM buffer o & 1 (a chain of 3 x K/8
//     MMAs).  Once it is complete, each thread loads its TMEM lane (its target's row of the
//     partial) and adds it to FP32 registers, then releases the buffer for offset o + 2.  The
//     tensor cores' accumulation rounds toward zero; short chains keep that bias at a few
//     units of 2^-24, and the sum over the 189 offsets is rounded to nearest.
//   epilogue: each thread writes its target's p^2 local coefficients from the registers.
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

// Shapes per order.  KS = K steps of 8 per offset, split into NCH chunks of (nearly) equal size.
template <int P>
struct TcCfg {
    static constexpr int PP = P * P;
    static constexpr int PR = (PP + 7) / 8 * 8;      // rows of the CUDA-core operator table
    static constexpr int KP = (PP + 7) / 8 * 8;      // K, padded to the MMA's K step
    static constexpr int NP = (PP + 15) / 16 * 16;   // N, padded to a multiple of 16
    static constexpr int KS = KP / 8;
    static constexpr int CKMAX = P == 10 ? 4 : (P == 8 ? 4 : (P == 6 ? 5 : 2));  // K steps per chunk (max)
    static constexpr int NCH = (KS + CKMAX - 1) / CKMAX;
    static constexpr int KCMAX = 8 * ((KS + NCH - 1) / NCH);  // K width of the largest chunk
    static constexpr int TM = 128;                   // targets per tile (MMA M)
    static constexpr int NSTAGE = P == 10 ? 3 : (P == 6 ? 3 : 4);
    static constexpr int TMEM_COLS = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : (2 * NP <= 128 ? 128 : 256));  // two accumulators
    static constexpr int A_FLOATS = TM * KCMAX;      // one of A_hi / A_lo
    static constexpr int STAGE_FLOATS = 2 * A_FLOATS + 2 * NP * KCMAX;
    static constexpr size_t kSmemBytes = (size_t)NSTAGE * STAGE_FLOATS * sizeof(float);
    static constexpr int BLOCK_FLOATS = 2 * NP * KCMAX;  // one (offset, chunk) block of the table
    static constexpr int NTHREADS = 160;
    static_assert(NP >= 16 && NP <= 256 && NP % 16 == 0, "MMA N");
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
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
    case 4: return (size_t)kM2LCodes * TcCfg<4>::NCH * TcCfg<4>::BLOCK_FLOATS;
    case 6: return (size_t)kM2LCodes * TcCfg<6>::NCH * TcCfg<6>::BLOCK_FLOATS;
    case 8: return (size_t)kM2LCodes * TcCfg<8>::NCH * TcCfg<8>::BLOCK_FLOATS;
    case 10: return (size_t)kM2LCodes * TcCfg<10>::NCH * TcCfg<10>::BLOCK_FLOATS;
    }
    return 0;
}

// (offset code, chunk) blocks: B_hi then B_lo, each [kw/4][NP][4] (canonical K-major layout
// of the N x kw operand chunk), rows n >= p^2 and columns k >= p^2 zero
template <int P>
__global__ void k_build_m2l_tc(const float *__restrict__ ops, float *__restrict__ tc)
{
    using C = TcCfg<P>;
    const int code = blockIdx.x, c = blockIdx.y;
    int k0, kw;
    chunk_range(c, C::KS, C::NCH, k0, kw);
    float *blk = tc + ((size_t)code * C::NCH + c) * C::BLOCK_FLOATS;
    for (int e = threadIdx.x; e < C::NP * kw; e += blockDim.x) {
        const int n = e / kw, kk = e % kw, k = k0 + kk;
        const float v = (n < C::PP && k < C::PP) ? ops[((size_t)code * C::PP + k) * C::PR + n] : 0.f;
        const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
        const int o = (kk >> 2) * C::NP * 4 + n * 4 + (kk & 3);
        blk[o] = hi;
        blk[C::NP * kw + o] = lo;
    }
}

void launch_build_m2l_tc(int P, const float *ops, float *tc, cudaStream_t s)
{
    switch (P) {
    case 4: k_build_m2l_tc<4><<<dim3(kM2LCodes, TcCfg<4>::NCH), 256, 0, s>>>(ops, tc); break;
    case 6: k_build_m2l_tc<6><<<dim3(kM2LCodes, TcCfg<6>::NCH), 256, 0, s>>>(ops, tc); break;
    case 8: k_build_m2l_tc<8><<<dim3(kM2LCodes, TcCfg<8>::NCH), 256, 0, s>>>(ops, tc); break;
    case 10: k_build_m2l_tc<10><<<dim3(kM2LCodes, TcCfg<10>::NCH), 256, 0, s>>>(ops, tc); break;
    }
    note_launches(1);
}

struct TcTiles {
    int L;
    int ntiles_level[kMaxLevel + 1];
};

template <int P>
__global__ void __launch_bounds__(160, 1)
    k_m2l_tc(TcTiles tiles, const int4 *__restrict__ tdesc, const int32_t *__restrict__ tlist,
             const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
             const uint32_t *__restrict__ m2l_offs, const int32_t *__restrict__ m2l_ids,
             const uint16_t *__restrict__ m2l_code, const float *__restrict__ optc, const float *__restrict__ M,
             float *__restrict__ Lc, int *status)
{
    using C = TcCfg<P>;
    constexpr int PP = C::PP, NP = C::NP, TM = C::TM, NSTAGE = C::NSTAGE, NCH = C::NCH;
    constexpr int S = 189 * NCH;
    constexpr uint32_t kIdesc = tc_idesc_tf32(TM, NP);

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
            mbar_init(&full_bar[st], 5);  // 4 producer warps + the operator copy's expect_tx
            mbar_init(&empty_bar[st], 1);  // one tcgen05.commit
            s_issued[st] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&drain_full[b], 1);   // tcgen05.commit after an offset's last MMA
            mbar_init(&drain_empty[b], 4);  // the 4 draining warps
        }
        mbar_init(&done_bar, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 4) tmem_alloc(&s_tmem, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < 4) {
        // ================= producers / drainers: one thread per target row =================
        const int r = tid;
        const int64_t g = target(r);
        uint32_t ptr = 0, pend = 0;
        if (g >= 0 && end[g] > begin[g]) {
            ptr = m2l_offs[g];
            pend = m2l_offs[g + 1];
        }
        // FP32 sum over offsets of the per-offset TMEM partials (each a chain of few MMAs)
        float acc[NP];
#pragma unroll
        for (int n = 0; n < NP; ++n) acc[n] = 0.f;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        auto drain = [&](int oc) -> bool {
            const int b = oc & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&drain_full[b], (oc >> 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) return false;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(b * NP + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(v[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drain_empty[b]);
            return true;
        };
        bool alive = true;
        const float *src = nullptr;
        for (int s = 0; s < S && alive; ++s) {
            const int st = s % NSTAGE, oc = s / NCH, c = s % NCH;
            if (s >= NSTAGE) {
                int ok = 1;
                if (lane == 0)
                    ok = mbar_wait_bounded(&empty_bar[st], ((s / NSTAGE) - 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    alive = false;
                    break;
                }
            }
            int k0, kw;
            chunk_range(c, C::KS, NCH, k0, kw);
            float *stage = tsm + (size_t)st * C::STAGE_FLOATS;
            float *Ahi = stage, *Alo = stage + C::A_FLOATS, *B = stage + 2 * C::A_FLOATS;
            const int code = c_tc_codes[tau][oc];
            if (warp == 0 && lane == 0) {
                const uint32_t bytes = 2u * NP * kw * 4u;
                mbar_expect_tx(&full_bar[st], bytes);
                tma_bulk_g2s(B, optc + ((size_t)code * NCH + c) * C::BLOCK_FLOATS, bytes, &full_bar[st]);
                s_issued[st] += 1;
            }
            if (c == 0) {
                src = nullptr;
                if (ptr < pend && (int)m2l_code[ptr] == code) {
                    src = M + (size_t)m2l_ids[ptr] * PP;
                    ++ptr;
                }
            }
            // gather this chunk of the source expansion, split into TF32 halves
            float4 v[C::KCMAX / 4];
#pragma unroll
            for (int j = 0; j < C::KCMAX / 4; ++j) {
                const int k = k0 + 4 * j;
                v[j] = (src && 4 * j < kw && k < PP) ? __ldg(reinterpret_cast<const float4 *>(src + k))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < C::KCMAX / 4; ++j) {
                if (4 * j >= kw) break;
                const float4 x = v[j];
                float4 h, l;
                h.x = tf32_rna(x.x);
                h.y = tf32_rna(x.y);
                h.z = tf32_rna(x.z);
                h.w = tf32_rna(x.w);
                l.x = tf32_rna(x.x - h.x);
                l.y = tf32_rna(x.y - h.y);
                l.z = tf32_rna(x.z - h.z);
                l.w = tf32_rna(x.w - h.w);
                *reinterpret_cast<float4 *>(Ahi + j * TM * 4 + r * 4) = h;
                *reinterpret_cast<float4 *>(Alo + j * TM * 4 + r * 4) = l;
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[st]);
            // the previous offset's partial is complete once this one is queued
            if (c == NCH - 1 && oc >= 1 && !drain(oc - 1)) alive = false;
        }
        if (alive && !drain(188)) alive = false;
        if (!alive && lane == 0) s_abort = 1;
        // every MMA has completed once done_bar has (bounded; needed before TMEM is freed)
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&done_bar, 0u, kWaitLimitNs, nullptr) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) s_abort = 1;
        __syncwarp();
        if (ok && alive && !s_abort && g >= 0 && end[g] > begin[g]) {
#pragma unroll
            for (int n = 0; n < PP; n += 4)
                *reinterpret_cast<float4 *>(Lc + g * PP + n) = make_float4(acc[n], acc[n + 1], acc[n + 2], acc[n + 3]);
        }
    } else if (lane == 0) {
        // ================= MMA issuer: offset oc accumulates in TMEM buffer oc & 1 =================
        for (int s = 0; s < S; ++s) {
            const int st = s % NSTAGE, oc = s / NCH, c = s % NCH, b = oc & 1;
            if (c == 0 && oc >= 2 &&
                !mbar_wait_bounded(&drain_empty[b], ((oc - 2) >> 1) & 1, kWaitLimitNs, &s_abort)) {
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
            const float *stage = tsm + (size_t)st * C::STAGE_FLOATS;
            const float *Ahi = stage, *Alo = stage + C::A_FLOATS;
            const float *Bhi = stage + 2 * C::A_FLOATS, *Blo = Bhi + NP * kw;
            const uint32_t d = tmem + (uint32_t)(b * NP);
            for (int j = 0; j < kw / 8; ++j) {
                const uint64_t ah = smem_desc(Ahi + j * 2 * TM * 4, TM * 16, 128);
                const uint64_t al = smem_desc(Alo + j * 2 * TM * 4, TM * 16, 128);
                const uint64_t bh = smem_desc(Bhi + j * 2 * NP * 4, NP * 16, 128);
                const uint64_t bl = smem_desc(Blo + j * 2 * NP * 4, NP * 16, 128);
                // the small cross terms first, the hi*hi term last
                tc_mma_tf32(d, al, bh, kIdesc, (c > 0 || j > 0) ? 1u : 0u);
                tc_mma_tf32(d, ah, bl, kIdesc, 1u);
                tc_mma_tf32(d, ah, bh, kIdesc, 1u);
            }
            tc_commit(&empty_bar[st]);
            if (c == NCH - 1) tc_commit(&drain_full[b]);
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
    if (warp == 4) {
        __syncwarp();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int P>
static void launch_m2l_tc_t(const TcTiles &tiles, int grid, const int4 *tdesc, const int32_t *tlist,
                            const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                            const int32_t *m2l_ids, const uint16_t *m2l_code, const float *optc, const float *M,
                            float *Lc, int *status, cudaStream_t s)
{
    using C = TcCfg<P>;
    cudaFuncSetAttribute(k_m2l_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmemBytes);
    k_m2l_tc<P><<<grid, C::NTHREADS, C::kSmemBytes, s>>>(tiles, tdesc, tlist, begin, end, m2l_offs, m2l_ids,
                                                          m2l_code, optc, M, Lc, status);
    note_launches(1);
}

static void dispatch_tc(int P, const TcTiles &tiles, int grid, const int4 *tdesc, const int32_t *tlist,
                        const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                        const uint16_t *m2l_code, const float *optc, const float *M, float *Lc, int *status,
                        cudaStream_t s)
{
    switch (P) {
    case 4: launch_m2l_tc_t<4>(tiles, grid, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s); break;
    case 6: launch_m2l_tc_t<6>(tiles, grid, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s); break;
    case 8: launch_m2l_tc_t<8>(tiles, grid, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s); break;
    case 10: launch_m2l_tc_t<10>(tiles, grid, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, optc, M, Lc, status, s); break;
    }
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

bool m2l_use_tc()
{
    static const bool on = [] {
        const char *e = getenv("GBFMM_M2L_TC");
        return !(e && atoi(e) == 0);
    }();
    return on;
}

}  // namespace gbfmm
