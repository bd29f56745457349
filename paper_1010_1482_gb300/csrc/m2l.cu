// M2L (Eq. 4) on the device as a batched FP32 contraction.
//
// With expansions scaled by the cell side, the translation from a source cell at integer
// offset o (in cells of the level) to the target is a fixed real p^2 x p^2 matrix T_o.  All
// targets with the same child position tau (key & 7) have the same 189 admissible offsets
// (children of the parent's neighbours that are not neighbours, Section "The M2L kernel
// implementation"), so a CTA takes TN targets of one level and one tau and walks those 189
// offsets in ascending code order, accumulating L~(:, targets) += T_o M~(:, sources).
//
// Warp specialisation: one producer warp keeps each target's CSR list pointer in registers,
// resolves the source of every target for the next offset, and stages T_o and the TN source
// expansions into a ring of NSTAGE shared-memory stages with TMA bulk copies (cp.async.bulk,
// completion on the stage's "full" mbarrier; a block of zeros stands in for missing sources).
// The consumer warps wait on "full", run a register-blocked FP32 micro-kernel (4 rows x CN
// targets per thread) and release the stage on its "empty" mbarrier.  No block-wide barrier
// runs inside the offset loop.  Every wait is bounded (1 s of %globaltimer); on timeout the
// kernel raises the status word, waits (bounded) for its copies in flight and returns.
#include "common.cuh"
#include "ptx.cuh"

#include <stdlib.h>

namespace gbfmm {

__constant__ uint16_t c_codes[8][189];

void init_m2l_constants()
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
    cudaMemcpyToSymbol(c_codes, codes, sizeof(codes));
}



// Exercises the bounded wait on its own: one thread waits on an mbarrier that no thread
// arrives on, gives up after limit_ns and raises the status word, as a pipeline stage whose
// copies never land would.
__global__ void k_wait_selftest(uint64_t limit_ns, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait_bounded(&bar, 0u, limit_ns, nullptr)) atomicOr(status, kStatusTimeout);
    }
}

void launch_wait_selftest(uint64_t limit_ns, int *status, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, status);
    note_launches(1);
}

struct M2LTiles {
    int L;
    int ntiles_level[kMaxLevel + 1];  // tiles of each level (levels processed L, L-1, ..., 2)
};

template <int P, int TN, int RM, int CN, int NSTAGE, int MINB>
struct M2LConfig {
    static constexpr int PP = P * P;
    static constexpr int PR = ops_rows_padded(P);
    static constexpr int SB = staged_col_stride(P);
    static constexpr int NRG = PR / RM;             // row groups
    static constexpr int NCG = TN / CN;             // column groups
    static constexpr int NCT = NRG * NCG;           // consumer threads with work
    static constexpr int NCW = (NCT + 31) / 32;     // consumer warps
    static constexpr int NTHREADS = NCW * 32 + 32;  // + one producer warp
    static constexpr int TPL = TN / 32;             // targets per producer lane
    static constexpr uint32_t kOpBytes = PP * PR * 4;
    static constexpr uint32_t kColBytes = PP * 4;
    static constexpr size_t kStageFloats = (size_t)PP * PR + (size_t)TN * SB;
    static constexpr size_t kSmemBytes = NSTAGE * kStageFloats * sizeof(float);
    static_assert(PR % RM == 0 && RM % 4 == 0 && TN % CN == 0 && TN % 32 == 0, "tile shape");
};

template <int P, int TN, int RM, int CN, int NSTAGE, int MINB>
__global__ void __launch_bounds__(M2LConfig<P, TN, RM, CN, NSTAGE, MINB>::NTHREADS, MINB)
    k_m2l(M2LTiles tiles, const int4 *__restrict__ tdesc, const int32_t *__restrict__ tlist,
          const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
          const uint32_t *__restrict__ m2l_offs, const int32_t *__restrict__ m2l_ids,
          const uint16_t *__restrict__ m2l_code, const float *__restrict__ ops, const float *__restrict__ M,
          float *__restrict__ Lc, const float *__restrict__ zero_block, int *status)
{
    using Cfg = M2LConfig<P, TN, RM, CN, NSTAGE, MINB>;
    constexpr int PP = Cfg::PP, PR = Cfg::PR, SB = Cfg::SB, NCG = Cfg::NCG, NCT = Cfg::NCT, NCW = Cfg::NCW;
    constexpr int S = 189;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stage_base = reinterpret_cast<float *>(smem_raw);  // NSTAGE x [A: PP*PR | B: TN*SB]
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE];
    __shared__ int s_issued[NSTAGE];
    __shared__ volatile int s_abort;

    // ---- decode tile ----
    // dense uniform levels (levels in descending order, target q of child position tau at
    // level_offset(l) + 8q + tau), or an explicit tile list (level, tau, start, count) over tlist
    int l, tau;
    int64_t q0 = 0, nq = 0, off = 0, tstart = 0;
    int tcount = 0;
    if (tdesc) {
        const int4 d = tdesc[blockIdx.x];
        if (d.w <= 0) return;  // an empty tile (the whole CTA, before any barrier)
        l = d.x;
        tau = d.y;
        tstart = d.z;
        tcount = d.w;
    } else {
        int rem = blockIdx.x;
        l = tiles.L;
        while (l >= 2 && rem >= tiles.ntiles_level[l]) {
            rem -= tiles.ntiles_level[l];
            --l;
        }
        if (l < 2) return;
        nq = int64_t(1) << (3 * (l - 1));
        const int64_t qtiles = (nq + TN - 1) / TN;
        tau = (int)(rem / qtiles);
        q0 = (rem % qtiles) * TN;
        off = level_offset(l);
    }
    // global cell index of tile target t, or -1
    auto target = [&](int t) -> int64_t {
        if (tdesc) return t < tcount ? (int64_t)tlist[tstart + t] : -1;
        const int64_t q = q0 + t;
        return q < nq ? off + 8 * q + tau : -1;
    };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int st = 0; st < NSTAGE; ++st) {
            mbar_init(&full_bar[st], 1);
            mbar_init(&empty_bar[st], NCW);
            s_issued[st] = 0;
        }
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NCW) {
        // ================= producer warp =================
        uint32_t ptr[Cfg::TPL], pend[Cfg::TPL];
#pragma unroll
        for (int k = 0; k < Cfg::TPL; ++k) {
            const int64_t g = target(lane + 32 * k);
            ptr[k] = pend[k] = 0;
            if (g >= 0) {
                if (end[g] > begin[g]) {
                    ptr[k] = m2l_offs[g];
                    pend[k] = m2l_offs[g + 1];
                }
            }
        }
        for (int s = 0; s < S; ++s) {
            const int st = s % NSTAGE;
            if (s >= NSTAGE) {
                const uint32_t parity = ((s / NSTAGE) - 1) & 1;
                int ok = 1;
                if (lane == 0) ok = mbar_wait_bounded(&empty_bar[st], parity, kWaitLimitNs, &s_abort) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) s_abort = 1;
                    break;
                }
            }
            const int code = c_codes[tau][s];
            const float *src_col[Cfg::TPL];
#pragma unroll
            for (int k = 0; k < Cfg::TPL; ++k) {
                const float *src = zero_block;
                if (ptr[k] < pend[k] && (int)m2l_code[ptr[k]] == code) {
                    src = M + (size_t)m2l_ids[ptr[k]] * PP;
                    ++ptr[k];
                }
                src_col[k] = src;
            }
            float *A = stage_base + st * Cfg::kStageFloats;
            float *B = A + PP * PR;
            if (lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(&full_bar[st], Cfg::kOpBytes + TN * Cfg::kColBytes);
                tma_bulk_g2s(A, ops + (size_t)code * PP * PR, Cfg::kOpBytes, &full_bar[st]);
                s_issued[st] += 1;
            }
            __syncwarp();
            fence_proxy_async();
#pragma unroll
            for (int k = 0; k < Cfg::TPL; ++k)
                tma_bulk_g2s(B + (lane + 32 * k) * SB, src_col[k], Cfg::kColBytes, &full_bar[st]);
        }
    } else {
        // ================= consumer warps =================
        constexpr int CNN = TN / NCG;
        const bool work = tid < NCT;
        const int cg = tid % NCG, rg = tid / NCG;
        float acc[RM][CNN];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < CNN; ++j) acc[i][j] = 0.f;
        for (int s = 0; s < S; ++s) {
            const int st = s % NSTAGE;
            const uint32_t parity = (s / NSTAGE) & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&full_bar[st], parity, kWaitLimitNs, &s_abort) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) s_abort = 1;
                break;
            }
            if (work) {
                const float *A = stage_base + st * Cfg::kStageFloats + rg * RM;
                const float *B = stage_base + st * Cfg::kStageFloats + PP * PR + cg * SB;
                // two k-groups per iteration: the compiler overlaps the second group's
                // fragment loads with the first group's FMAs
#pragma unroll 2
                for (int k = 0; k < PP; k += 4) {
                    Frag<CNN, RM> f;
                    f.load(A, B, k, PR, NCG * SB);
                    f.fma(acc);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[st]);
        }
        if (work && !s_abort) {
#pragma unroll
            for (int j = 0; j < CNN; ++j) {
                const int64_t g = target(cg + j * NCG);
                if (g < 0) continue;
                if (end[g] <= begin[g]) continue;
#pragma unroll
                for (int qq = 0; qq < RM / 4; ++qq) {
                    const int r = rg * RM + 4 * qq;
                    if (r < PP)
                        *reinterpret_cast<float4 *>(Lc + g * PP + r) = make_float4(
                            acc[4 * qq][j], acc[4 * qq + 1][j], acc[4 * qq + 2][j], acc[4 * qq + 3][j]);
                }
            }
        }
    }
    __syncthreads();
    if (s_abort) {
        // let every issued copy land before the CTA's shared memory is released (bounded)
        if (tid == 0) {
            atomicOr(status, kStatusTimeout);
            for (int st = 0; st < NSTAGE; ++st)
                if (s_issued[st] > 0) mbar_wait_bounded(&full_bar[st], (s_issued[st] - 1) & 1, kWaitLimitNs, nullptr);
        }
        __syncthreads();
    }
}

template <int P, int TN, int RM, int CN, int NSTAGE, int MINB>
static void launch_m2l_t(int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                         const int32_t *m2l_ids, const uint16_t *m2l_code, const float *ops, const float *M,
                         float *Lc, const float *zero_block, int *status, cudaStream_t s)
{
    using Cfg = M2LConfig<P, TN, RM, CN, NSTAGE, MINB>;
    cudaFuncSetAttribute(k_m2l<P, TN, RM, CN, NSTAGE, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Cfg::kSmemBytes);
    M2LTiles tiles{};
    tiles.L = L;
    int total = 0;
    for (int l = 2; l <= L; ++l) {
        int64_t nq = int64_t(1) << (3 * (l - 1));
        tiles.ntiles_level[l] = (int)(8 * ((nq + TN - 1) / TN));
        total += tiles.ntiles_level[l];
    }
    if (total == 0) return;
    k_m2l<P, TN, RM, CN, NSTAGE, MINB><<<total, Cfg::NTHREADS, Cfg::kSmemBytes, s>>>(
        tiles, nullptr, nullptr, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status);
    note_launches(1);
}

// tile-list mode (adaptive tree): the default tile shape, kM2LTargetsPerTile targets per CTA
template <int P, int NSTAGE>
static void launch_m2l_tiles_t(const int4 *tdesc, int ntiles, const int32_t *tlist, const int32_t *begin,
                               const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                               const uint16_t *m2l_code, const float *ops, const float *M, float *Lc,
                               const float *zero_block, int *status, cudaStream_t s)
{
    constexpr int TN = kM2LTargetsPerTile;
    using Cfg = M2LConfig<P, TN, 4, 8, NSTAGE, 1>;
    cudaFuncSetAttribute(k_m2l<P, TN, 4, 8, NSTAGE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Cfg::kSmemBytes);
    M2LTiles tiles{};
    k_m2l<P, TN, 4, 8, NSTAGE, 1><<<ntiles, Cfg::NTHREADS, Cfg::kSmemBytes, s>>>(
        tiles, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status);
    note_launches(1);
}

void launch_m2l_tiles(int P, const int4 *tdesc, int ntiles, const int32_t *tlist, const int32_t *begin,
                      const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids, const uint16_t *m2l_code,
                      const float *ops, const float *M, float *Lc, const float *zero_block, int *status,
                      cudaStream_t s)
{
    if (ntiles <= 0) return;
    switch (P) {
    case 4: launch_m2l_tiles_t<4, 4>(tdesc, ntiles, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    case 6: launch_m2l_tiles_t<6, 4>(tdesc, ntiles, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    case 8: launch_m2l_tiles_t<8, 4>(tdesc, ntiles, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    case 10: launch_m2l_tiles_t<10, 3>(tdesc, ntiles, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    }
}

void launch_m2l(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                const int32_t *m2l_ids, const uint16_t *m2l_code, const float *ops, const float *M, float *Lc,
                const float *zero_block, int *status, cudaStream_t s)
{
    if (L < 2) return;
#define GBFMM_M2L_ARGS L, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s
    // 64 targets per CTA, 4 operator rows x 8 targets per thread
    switch (P) {
    case 4: launch_m2l_t<4, 64, 4, 8, 4, 1>(GBFMM_M2L_ARGS); break;
    case 6: launch_m2l_t<6, 64, 4, 8, 4, 1>(GBFMM_M2L_ARGS); break;
    case 8: launch_m2l_t<8, 64, 4, 8, 4, 1>(GBFMM_M2L_ARGS); break;
    case 10: launch_m2l_t<10, 64, 4, 8, 3, 1>(GBFMM_M2L_ARGS); break;
    }
#undef GBFMM_M2L_ARGS
}

}  // namespace gbfmm
