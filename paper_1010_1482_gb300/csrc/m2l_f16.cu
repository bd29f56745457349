// M2L (Eq. 4) over interaction lists on the tcgen05 tensor cores: the adaptive tree's V lists
// (and the uniform tree's M2L lists with GBFMM_FLAG_M2L_GATHERED).  FP16 operands split in three
// products ("3xF16"), FP32 accumulation.  A CTA takes 128 target cells of one level and one child
// position tau (the MMA's M); they share the 189 admissible offsets, walked in stencil-code order:
// D[128 x p^2] += A[128 x K] (the targets' gathered source expansions, in TMEM) . T_o^T (one
// offset's operator, in shared memory); each offset's partial is drained to FP32 registers.
//
// Range: FP16 has a 5-bit exponent, so both operands are brought to a fixed magnitude by exact
// power-of-two scales: each offset's operator by 2^g_o (max |T_o| -> 2^12, chosen when the
// table is built) and each source expansion by 2^s_c (max |M~_c| -> 2^10, one byte per cell,
// computed after the upward pass).  The drain multiplies each offset's partial by
// 2^-(g_o + s_c) before adding it in FP32.  hi = fp16(x), lo = fp16(x - hi): the products
// hi*hi + lo*hi + hi*lo carry 22 significant bits of each operand; entries far below an
// operand's maximum lose relative precision in FP16's subnormal range, but their products are
// below 2^-24 of the largest ones.
#include "common.cuh"
#include "ptx.cuh"

#include <cuda_fp16.h>

namespace gbfmm {

__constant__ uint16_t c_f16_codes[8][189];

void init_m2l_f16_constants()
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
    cudaMemcpyToSymbol(c_f16_codes, codes, sizeof(codes));
}

// 2^e as a float (e within the normal range)
GB_DEV float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// ---- operator table: per code T_hi then T_lo (FP16), each [KP/8][NP][8] (the canonical
// no-swizzle K-major layout of the N x K operand, 8 halves per 16-byte row), scaled by 2^g_o;
// g_o at the end of the table -----------------------------------------------------------------
template <int P>
struct F16Table {
    static constexpr int PP = P * P, PR = (PP + 7) / 8 * 8, KP = (PP + 15) / 16 * 16, NP = (PP + 15) / 16 * 16;
    static constexpr int HALF = KP * NP;          // halves of T_hi (or T_lo)
    static constexpr int CODE_HALVES = 2 * HALF;
};

size_t m2l_f16_table_bytes(int P)
{
    size_t h = 0;
    switch (P) {
    case 4: h = F16Table<4>::CODE_HALVES; break;
    case 6: h = F16Table<6>::CODE_HALVES; break;
    case 8: h = F16Table<8>::CODE_HALVES; break;
    case 10: h = F16Table<10>::CODE_HALVES; break;
    }
    return (size_t)kM2LCodes * h * 2 + (size_t)kM2LCodes * sizeof(int);
}

template <int P>
__global__ void __launch_bounds__(256) k_build_m2l_f16(const float *__restrict__ ops, __half *__restrict__ tab,
                                                        int *__restrict__ gexp)
{
    using T = F16Table<P>;
    const int code = blockIdx.x;
    const float *src = ops + (size_t)code * T::PP * T::PR;  // [k][row], rows padded to PR
    __shared__ float s_red[8];
    float m = 0.f;
    for (int e = threadIdx.x; e < T::PP * T::PP; e += blockDim.x) m = fmaxf(m, fabsf(src[(e / T::PP) * T::PR + e % T::PP]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_red[w]);
    int ex = 0;
    if (m > 0.f) frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
    const int g = m > 0.f ? 12 - ex : 0;
    if (threadIdx.x == 0) gexp[code] = g;
    const float sc = pow2f(g);
    __half *blk = tab + (size_t)code * T::CODE_HALVES;
    for (int e = threadIdx.x; e < T::NP * T::KP; e += blockDim.x) {
        const int n = e / T::KP, k = e % T::KP;
        const float v = (n < T::PP && k < T::PP) ? src[(size_t)k * T::PR + n] * sc : 0.f;
        const __half hi = __float2half_rn(v);
        const __half lo = __float2half_rn(v - __half2float(hi));
        const int o = (k >> 3) * T::NP * 8 + n * 8 + (k & 7);
        blk[o] = hi;
        blk[T::HALF + o] = lo;
    }
}

void launch_build_m2l_f16(int P, const float *ops, void *table, cudaStream_t s)
{
    __half *tab = static_cast<__half *>(table);
    switch (P) {
    case 4: k_build_m2l_f16<4><<<kM2LCodes, 256, 0, s>>>(ops, tab, reinterpret_cast<int *>(tab + (size_t)kM2LCodes * F16Table<4>::CODE_HALVES)); break;
    case 6: k_build_m2l_f16<6><<<kM2LCodes, 256, 0, s>>>(ops, tab, reinterpret_cast<int *>(tab + (size_t)kM2LCodes * F16Table<6>::CODE_HALVES)); break;
    case 8: k_build_m2l_f16<8><<<kM2LCodes, 256, 0, s>>>(ops, tab, reinterpret_cast<int *>(tab + (size_t)kM2LCodes * F16Table<8>::CODE_HALVES)); break;
    case 10: k_build_m2l_f16<10><<<kM2LCodes, 256, 0, s>>>(ops, tab, reinterpret_cast<int *>(tab + (size_t)kM2LCodes * F16Table<10>::CODE_HALVES)); break;
    }
    note_launches(1);
}

// ---- shapes of the list-based kernel --------------------------------------------------------
template <int P>
struct F16Cfg {
    static constexpr int PP = P * P;
    static constexpr int KP = (PP + 15) / 16 * 16;   // K, padded to the MMA's K step (16)
    static constexpr int NP = (PP + 15) / 16 * 16;   // N
    static constexpr int KS = KP / 16;
    static_assert(NP % 16 == 0 && NP <= 128, "MMA N");
};

GB_DEV void chunk16(int c, int KS, int NCH, int &k0, int &kw)
{
    const int s0 = (c * KS) / NCH, s1 = ((c + 1) * KS) / NCH;
    k0 = 16 * s0;
    kw = 16 * (s1 - s0);
}

struct F16Tiles {
    int L;
    int tile0;  // tile of block 0 (a launch may cover a range of the tiles)
    int ntiles_level[kMaxLevel + 1];
};

// ---- pre-split sources ------------------------------------------------------------------
// The sources can be converted once per cell instead of once per (target, offset): after the
// upward pass every cell's expansion is scaled by 2^s_c and split into FP16 halves, stored per
// piece of 8 coefficients as 8 hi halves then 8 lo halves (KP / 8 pieces, zero-padded), so a
// converter thread's hi and lo halves of a chunk are one contiguous 128-byte line.  With them
// the converter warps only load their target's source and store it into TMEM (the same bits
// the conversion produces, so the result is identical).
// one warp per cell
template <int P>
__global__ void __launch_bounds__(256) k_presplit(const float *__restrict__ M, Span cells,
                                                  int8_t *__restrict__ scale, __half *__restrict__ ps)
{
    constexpr int PP = P * P, KP = F16Cfg<P>::KP, PER = (KP + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= span_count(cells)) return;
    const int64_t c = span_first(cells) + w;
    float v[PER];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int k = lane + 32 * i;
        v[i] = k < PP ? M[c * PP + k] : 0.f;
        m = fmaxf(m, fabsf(v[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // the source scale: max |M~_c| = f 2^e, f in [0.5, 1) -> s_c = 10 - e
    const bool fin = m > 0.f && m <= 3.0e38f;
    int ex = 0;
    if (fin) frexpf(m, &ex);
    int sc = fin ? 10 - ex : 0;
    sc = sc < -100 ? -100 : (sc > 100 ? 100 : sc);
    if (lane == 0) scale[c] = (int8_t)sc;
    const float up = pow2f(sc);
    __half *row = ps + c * (2 * KP);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int k = lane + 32 * i;
        if (k < KP) {
            const float x = v[i] * up;
            const __half hi = __float2half_rn(x);
            row[(k >> 3) * 16 + (k & 7)] = hi;
            row[(k >> 3) * 16 + 8 + (k & 7)] = __float2half_rn(x - __half2float(hi));
        }
    }
}

size_t presplit_bytes(int P, int64_t ncells)
{
    const int KP = (P * P + 15) / 16 * 16;
    return (size_t)ncells * 4 * KP;
}

// cells: the cells to split (default: all ncells of them, counted on the host)
void launch_presplit(int P, const float *M, int64_t ncells, int8_t *scale, void *ps, cudaStream_t s, Span cells)
{
    if (cells.cap == 0 && !cells.dhi) cells = host_span(0, ncells);
    if (cells.cap <= 0) return;
    const unsigned grid = (unsigned)((cells.cap + 7) / 8);
    __half *h = static_cast<__half *>(ps);
    switch (P) {
    case 4: k_presplit<4><<<grid, 256, 0, s>>>(M, cells, scale, h); break;
    case 6: k_presplit<6><<<grid, 256, 0, s>>>(M, cells, scale, h); break;
    case 8: k_presplit<8><<<grid, 256, 0, s>>>(M, cells, scale, h); break;
    case 10: k_presplit<10><<<grid, 256, 0, s>>>(M, cells, scale, h); break;
    }
    note_launches(1);
}

// ---- staged variant: coalesced copies of the pre-split sources --------------------------------
// The converter warps' scattered 16-byte loads (every lane a different source row) kept the L1
// data pipe near its peak while the tensor pipe idled.  Here each converter warp first copies
// the chunk pieces of its 32 rows into a warp-private shared-memory slot with cp.async, 8 lanes
// per row (each instruction reads 4 rows x 128 contiguous bytes of the pre-split sources: 8 hi
// then 8 lo halves per 8 coefficients), one step ahead; then every lane reads its own row back
// (conflict-free 16-byte shared loads) and stores it into TMEM.  Only warp-local
// synchronisation: a warp reads only what it copied.
template <int P, int CW_>
struct F16SCfg {
    static constexpr int PP = P * P, KP = F16Cfg<P>::KP, NP = F16Cfg<P>::NP, KS = KP / 16;
    static constexpr int NCH = (KS + 3) / 4, TM = 128, CW = CW_;
    static constexpr int HW = CW / 4;                         // converter warps per TMEM lane quadrant
    static constexpr int SEG = 64 / HW;                       // halves of a chunk per warp
    static constexpr int UPR = SEG / 4;                       // 16-byte units per row (hi + lo)
    static constexpr int RSW = 4 * SEG + 16;                  // bytes per staged row (padded)
    static constexpr int SLOT_BYTES = 32 * RSW;               // one warp, one step
    static constexpr int STAGING_BYTES = CW * 2 * SLOT_BYTES; // two slots per warp
    static constexpr int B_BYTES = 2 * NP * 64 * 2;           // operator: B_hi | B_lo
    static constexpr int NSTAGE = STAGING_BYTES + 4 * B_BYTES <= 210 * 1024 ? 4 : 3;
    static constexpr size_t kBytes = (size_t)NSTAGE * B_BYTES + STAGING_BYTES;
    static constexpr size_t kSmemBytes = kBytes > 116 * 1024 ? kBytes : 116 * 1024;
    static constexpr int TMEM_COLS = 512, A_COL0 = 256;      // D ping-pong, then A stages (64 columns each)
    static constexpr int NTHREADS = 32 * (CW + 1);
    static constexpr int NH = NP / HW;                        // output columns drained per thread
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
    static_assert(A_COL0 + 64 * NSTAGE <= TMEM_COLS, "TMEM A stages");
    static_assert(B_BYTES % 1024 == 0, "stage alignment");
    static_assert(NH % 4 == 0 && SEG % 8 == 0, "converter split");
};

template <int P, int CW_>
__global__ void __launch_bounds__(F16SCfg<P, CW_>::NTHREADS, 1)
    k_m2l_f16s(F16Tiles tiles, const int4 *__restrict__ tdesc, const int32_t *__restrict__ tlist,
               const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
               const uint32_t *__restrict__ m2l_offs, const int32_t *__restrict__ m2l_ids,
               const uint16_t *__restrict__ m2l_code, const __half *__restrict__ tab, const int *__restrict__ gexp,
               const __half *__restrict__ ps, const int8_t *__restrict__ cscale, float *__restrict__ Lc, int *status)
{
    using C = F16SCfg<P, CW_>;
    using T = F16Table<P>;
    constexpr int PP = C::PP, KP = C::KP, NP = C::NP, NH = C::NH, TM = C::TM, NSTAGE = C::NSTAGE, NCH = C::NCH;
    constexpr int S = 189 * NCH, CW = C::CW, SEG = C::SEG, UPR = C::UPR;
    constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);  // F32 += F16 x F16
    constexpr int kMmaWarp = CW;

    extern __shared__ __align__(1024) unsigned char f16ssm[];
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], drain_full[2], drain_empty[2], done_bar;
    __shared__ int s_issued[NSTAGE];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    int tau;
    int64_t q0 = 0, nq = 0, off = 0, tstart = 0;
    int tcount = 0;
    if (tdesc) {
        const int4 d = tdesc[tiles.tile0 + blockIdx.x];
        if (d.w <= 0) return;  // an empty tile (the whole CTA, before any barrier or TMEM)
        tau = d.y;
        tstart = d.z;
        tcount = d.w;
    } else {
        int rem = tiles.tile0 + blockIdx.x;
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
            mbar_init(&full_bar[st], CW + 1);  // the converter warps + the operator copies' expect_tx
            mbar_init(&empty_bar[st], 1);      // one tcgen05.commit
            s_issued[st] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&drain_full[b], 1);
            mbar_init(&drain_empty[b], CW);
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
    unsigned char *bstages = f16ssm;
    unsigned char *staging = f16ssm + (size_t)NSTAGE * C::B_BYTES;

    if (warp < CW) {
        // ===== converters / drainers: target row r; halves [SEG h, SEG h + SEG) of each chunk;
        // output columns [h NH, h NH + NH) =====
        const int quad = warp & 3, h = warp >> 2;
        const int r = 32 * quad + lane;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        const int64_t g = target(r);
        uint32_t ptr = 0, pend = 0;
        if (g >= 0 && end[g] > begin[g]) {
            ptr = m2l_offs[g];
            pend = m2l_offs[g + 1];
        }
        int nxt_code = 0xffff, nxt_id = 0;
        if (ptr < pend) {
            nxt_code = m2l_code[ptr];
            nxt_id = m2l_ids[ptr];
        }
        float acc[NH];
#pragma unroll
        for (int n = 0; n < NH; ++n) acc[n] = 0.f;
        auto drain = [&](int oc, float factor) -> bool {
            const int b = oc & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(&drain_full[b], (oc >> 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) return false;
            tc_fence_after();
            // all the row's columns in flight at once, one wait
            static_assert(NH % 8 == 0, "drain in 8-column loads");
            uint32_t v[NH];
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += 8) tmem_ld8_nowait(tmem + lane_base + (uint32_t)(b * NP + h * NH + c0), v + c0);
            tmem_wait_ld_regs(v);
#pragma unroll
            for (int n = 0; n < NH; ++n) acc[n] = fmaf(__uint_as_float(v[n]), factor, acc[n]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drain_empty[b]);
            return true;
        };
        // copies of step s2 into slot s2 & 1: this warp's 32 rows, UPR lanes per row (16 bytes
        // each: unit u = 2 i + {hi, lo} of coefficient piece SEG h / 8 + i); the offset's source
        // and unscaling factor are taken from the list at its first chunk
        const __half *mysrc = ps;
        int myok = 0;
        float fac[2] = {0.f, 0.f};
        auto issue = [&](int s2) {
            const int oc2 = s2 / NCH, c2 = s2 % NCH;
            if (c2 == 0) {
                const int code = c_f16_codes[tau][oc2];
                myok = 0;
                float f = 0.f;
                if (nxt_code == code) {
                    mysrc = ps + (size_t)nxt_id * (2 * KP);
                    myok = 1;
                    f = pow2f(-((int)cscale[nxt_id] + gexp[code]));
                    ++ptr;
                    nxt_code = 0xffff;
                    if (ptr < pend) {
                        nxt_code = m2l_code[ptr];
                        nxt_id = m2l_ids[ptr];
                    }
                }
                if (oc2 & 1)
                    fac[1] = f;
                else
                    fac[0] = f;
            }
            int k0, kw;
            chunk16(c2, C::KS, NCH, k0, kw);
            unsigned char *slot = staging + (size_t)(warp * 2 + (s2 & 1)) * C::SLOT_BYTES;
            const int u = lane % UPR;
            const bool uok = SEG * h + 8 * (u >> 1) < kw;
#pragma unroll
            for (int it = 0; it < UPR; ++it) {
                const int rl = (32 / UPR) * it + lane / UPR;
                const __half *sp = reinterpret_cast<const __half *>(
                    __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(mysrc), rl));
                const int ok = __shfl_sync(0xffffffffu, myok, rl);
                cp_async16(slot + (size_t)rl * C::RSW + 16 * u, sp + 2 * k0 + 2 * SEG * h + 8 * u,
                           (ok && uok) ? 16u : 0u);
            }
            cp_async_commit();
        };
        bool alive = true;
        float pend_factor = 0.f;
        issue(0);
        for (int s = 0; s < S && alive; ++s) {
            const int st = s % NSTAGE, oc = s / NCH, c = s % NCH;
            const float cur_factor = (oc & 1) ? fac[1] : fac[0];
            if (s + 1 < S) {
                issue(s + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            uint32_t hi[SEG / 2], lo[SEG / 2];
            const uint4 *rp = reinterpret_cast<const uint4 *>(staging + (size_t)(warp * 2 + (s & 1)) * C::SLOT_BYTES +
                                                              (size_t)lane * C::RSW);
#pragma unroll
            for (int i = 0; i < SEG / 8; ++i) {
                const uint4 a = rp[2 * i], b = rp[2 * i + 1];
                hi[4 * i] = a.x;
                hi[4 * i + 1] = a.y;
                hi[4 * i + 2] = a.z;
                hi[4 * i + 3] = a.w;
                lo[4 * i] = b.x;
                lo[4 * i + 1] = b.y;
                lo[4 * i + 2] = b.z;
                lo[4 * i + 3] = b.w;
            }
            __syncwarp();  // the slot is refilled by the next step's copies
            if (s >= NSTAGE) {
                int ok = 1;
                if (lane == 0)
                    ok = mbar_wait_bounded(&empty_bar[st], ((s / NSTAGE) - 1) & 1, kWaitLimitNs, &s_abort) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    alive = false;
                    break;
                }
            }
            int k0, kw;
            chunk16(c, C::KS, NCH, k0, kw);
            if (tid == 0) {
                const uint32_t half = (uint32_t)NP * kw * 2u;
                const int code = c_f16_codes[tau][oc];
                const __half *tb = tab + (size_t)code * T::CODE_HALVES + (size_t)k0 * NP;
                __half *B = reinterpret_cast<__half *>(bstages + (size_t)st * C::B_BYTES);
                mbar_expect_tx(&full_bar[st], 2u * half);
                tma_bulk_g2s(B, tb, half, &full_bar[st]);
                tma_bulk_g2s(B + NP * kw, tb + T::HALF, half, &full_bar[st]);
                s_issued[st] += 1;
            }
            const uint32_t acol = (uint32_t)(C::A_COL0 + 64 * st + (SEG / 2) * h);
            tmem_st_cols<SEG / 2>(tmem + lane_base + acol, hi);
            tmem_st_cols<SEG / 2>(tmem + lane_base + acol + 32, lo);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[st]);
            // the previous offset's partial is complete once this one is queued
            if (c == NCH - 1 && oc >= 1 && !drain(oc - 1, pend_factor)) alive = false;
            if (c == NCH - 1) pend_factor = cur_factor;
        }
        cp_async_wait<0>();
        if (alive && !drain(188, pend_factor)) alive = false;
        if (!alive && lane == 0) s_abort = 1;
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
            chunk16(c, C::KS, NCH, k0, kw);
            const __half *Bhi = reinterpret_cast<const __half *>(bstages + (size_t)st * C::B_BYTES), *Blo = Bhi + NP * kw;
            const uint32_t d = tmem + (uint32_t)(b * NP);
            const uint32_t ahi = tmem + (uint32_t)(C::A_COL0 + 64 * st), alo = ahi + 32;
            for (int j = 0; j < kw / 16; ++j) {
                const uint64_t bh = smem_desc(Bhi + j * 2 * NP * 8, NP * 16, 128);
                const uint64_t bl = smem_desc(Blo + j * 2 * NP * 8, NP * 16, 128);
                tc_mma_f16_ta(d, alo + 8 * j, bh, kIdesc, (c > 0 || j > 0) ? 1u : 0u);
                tc_mma_f16_ta(d, ahi + 8 * j, bl, kIdesc, 1u);
                tc_mma_f16_ta(d, ahi + 8 * j, bh, kIdesc, 1u);
            }
            tc_commit(&empty_bar[st]);
            if (c == NCH - 1) tc_commit(&drain_full[b]);
        }
        tc_commit(&done_bar);
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

template <int P>
static void launch_f16_t(const F16Tiles &tiles, int grid, const int4 *tdesc, const int32_t *tlist, const int32_t *begin,
                         const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids, const uint16_t *m2l_code,
                         const void *table, const float *M, const int8_t *cscale, const void *ps, float *Lc,
                         int *status, cudaStream_t s, int max_ctas)
{
    using T = F16Table<P>;
    const __half *tab = static_cast<const __half *>(table);
    const int *gexp = reinterpret_cast<const int *>(tab + (size_t)kM2LCodes * T::CODE_HALVES);
    using CS = F16SCfg<P, 8>;
    cudaFuncSetAttribute(k_m2l_f16s<P, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CS::kSmemBytes);
    const int step = max_ctas > 0 ? max_ctas : grid;
    for (int t0 = 0; t0 < grid; t0 += step) {
        F16Tiles tt = tiles;
        tt.tile0 = t0;
        const int g = grid - t0 < step ? grid - t0 : step;
        k_m2l_f16s<P, 8><<<g, CS::NTHREADS, CS::kSmemBytes, s>>>(tt, tdesc, tlist, begin, end, m2l_offs, m2l_ids,
                                                                 m2l_code, tab, gexp, static_cast<const __half *>(ps),
                                                                 cscale, Lc, status);
        note_launches(1);
    }
}

// ps: the pre-split sources (launch_presplit)
static void dispatch_f16(int P, const F16Tiles &tiles, int grid, const int4 *tdesc, const int32_t *tlist,
                         const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                         const uint16_t *m2l_code, const void *table, const float *M, const int8_t *cscale,
                         const void *ps, float *Lc, int *status, cudaStream_t s, int max_ctas)
{
#define GBFMM_F16_ARGS tiles, grid, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, table, M, cscale, ps, Lc, status, s, max_ctas
    switch (P) {
    case 4: launch_f16_t<4>(GBFMM_F16_ARGS); break;
    case 6: launch_f16_t<6>(GBFMM_F16_ARGS); break;
    case 8: launch_f16_t<8>(GBFMM_F16_ARGS); break;
    case 10: launch_f16_t<10>(GBFMM_F16_ARGS); break;
    }
#undef GBFMM_F16_ARGS
}

void launch_m2l_f16(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                    const int32_t *m2l_ids, const uint16_t *m2l_code, const void *table, const float *M,
                    const int8_t *cscale, const void *ps, float *Lc, int *status, cudaStream_t s, int max_ctas)
{
    if (L < 2) return;
    F16Tiles tiles{};
    tiles.L = L;
    int total = 0;
    for (int l = 2; l <= L; ++l) {
        const int64_t nq = int64_t(1) << (3 * (l - 1));
        tiles.ntiles_level[l] = (int)(8 * ((nq + kM2LTcTargetsPerTile - 1) / kM2LTcTargetsPerTile));
        total += tiles.ntiles_level[l];
    }
    if (total == 0) return;
    dispatch_f16(P, tiles, total, nullptr, nullptr, begin, end, m2l_offs, m2l_ids, m2l_code, table, M, cscale, ps, Lc,
                 status, s, max_ctas);
}

void launch_m2l_f16_tiles(int P, const int4 *tdesc, int ntiles, const int32_t *tlist, const int32_t *begin,
                          const int32_t *end, const uint32_t *m2l_offs, const int32_t *m2l_ids,
                          const uint16_t *m2l_code, const void *table, const float *M, const int8_t *cscale,
                          const void *ps, float *Lc, int *status, cudaStream_t s, int max_ctas)
{
    if (ntiles <= 0) return;
    F16Tiles tiles{};
    dispatch_f16(P, tiles, ntiles, tdesc, tlist, begin, end, m2l_offs, m2l_ids, m2l_code, table, M, cscale, ps, Lc,
                 status, s, max_ctas);
}

}  // namespace gbfmm
