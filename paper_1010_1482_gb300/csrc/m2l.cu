// M2L (Eq. 4) on the device as a batched FP32 contraction.
//
// With expansions scaled by the cell side, the translation from a source cell at integer
// offset o (in cells of the level) to the target is a fixed real p^2 x p^2 matrix T_o.  All
// targets with the same child position tau (key & 7) have the same 189 admissible offsets
// (children of the parent's neighbours that are not neighbours, Section "The M2L kernel
// implementation"), so a CTA takes TN targets of one level and one tau and walks those 189
// offsets in ascending code order; for each it stages T_o and the TN source expansions (one
// per target, read through the target's CSR list row) in shared memory with TMA bulk copies
// (double-buffered, mbarrier completion), and accumulates L~(:, targets) += T_o M~(:, sources)
// with a register-blocked FP32 micro-kernel (RM rows x CN targets per thread).
// Missing sources (domain boundary, empty cells) are copied from a block of zeros.
// Every mbarrier wait is bounded; on timeout the kernel raises the status word and the CTA
// stops after a second bounded wait for its copies in flight.
#include "common.cuh"

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

// ---- PTX wrappers -------------------------------------------------------------------------
GB_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

GB_DEV void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

GB_DEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

GB_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

GB_DEV void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

GB_DEV void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

GB_DEV bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

GB_DEV uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: true on completion, false after ~limit_ns.
GB_DEV bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

// stride (floats) of one staged source column: a multiple of 4 with (stride / 4) odd, so the
// 16-byte column reads of eight consecutive targets fall in distinct bank groups
template <int P>
struct M2LShape {
    static constexpr int PP = P * P;
    static constexpr int SB = ((PP / 4) % 2 == 1) ? PP : PP + 4;
};

struct M2LTiles {
    int L;
    int ntiles_level[kMaxLevel + 1];  // tiles of each level (levels processed L, L-1, ..., 2)
};

template <int P, int TN, int RM, int CN>
__global__ void __launch_bounds__((P * P / RM) * (TN / CN))
    k_m2l(M2LTiles tiles, const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
          const uint32_t *__restrict__ m2l_offs, const int32_t *__restrict__ m2l_ids,
          const uint16_t *__restrict__ m2l_code, const float *__restrict__ ops, const float *__restrict__ M,
          float *__restrict__ Lc, const float *__restrict__ zero_block, int *status)
{
    constexpr int PP = P * P;
    constexpr int SB = M2LShape<P>::SB;
    constexpr int NCG = TN / CN;
    constexpr int NTH = (PP / RM) * NCG;
    constexpr uint32_t kOpBytes = PP * PP * 4;
    constexpr uint32_t kColBytes = PP * 4;
    static_assert(PP % RM == 0 && TN % CN == 0 && RM == 4, "tile shape");
    static_assert(NTH >= TN, "one resolving thread per target");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sA = reinterpret_cast<float *>(smem_raw);  // [2][PP*PP]  operator, column-major
    float *sB = sA + 2 * PP * PP;                     // [2][TN*SB]  source columns
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_src[2][TN];
    __shared__ uint32_t s_ptr[TN], s_end[TN];
    __shared__ int s_abort;

    // ---- decode tile: levels in descending order ----
    int rem = blockIdx.x, l = tiles.L;
    while (l >= 2 && rem >= tiles.ntiles_level[l]) {
        rem -= tiles.ntiles_level[l];
        --l;
    }
    if (l < 2) return;
    const int64_t nq = int64_t(1) << (3 * (l - 1));
    const int64_t qtiles = (nq + TN - 1) / TN;
    const int tau = (int)(rem / qtiles);
    const int64_t q0 = (rem % qtiles) * TN;
    const int64_t off = level_offset(l);
    const int tid = threadIdx.x;

    if (tid < TN) {
        int64_t q = q0 + tid;
        uint32_t a = 0, b = 0;
        if (q < nq) {
            int64_t g = off + 8 * q + tau;
            if (end[g] > begin[g]) {
                a = m2l_offs[g];
                b = m2l_offs[g + 1];
            }
        }
        s_ptr[tid] = a;
        s_end[tid] = b;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // resolve the source of every target for slot s (threads < TN), into s_src[buf]
    auto resolve = [&](int s, int buf) {
        if (tid < TN) {
            const int code = c_codes[tau][s];
            uint32_t pidx = s_ptr[tid];
            int src = -1;
            if (pidx < s_end[tid] && (int)m2l_code[pidx] == code) {
                src = m2l_ids[pidx];
                s_ptr[tid] = pidx + 1;
            }
            s_src[buf][tid] = src;
        }
    };
    // issue the copies of slot s into buffer buf (after a barrier that published s_src[buf])
    auto issue = [&](int s, int buf) {
        if (tid == 0) {
            fence_proxy_async();
            mbar_expect_tx(&bar[buf], kOpBytes + TN * kColBytes);
            const int code = c_codes[tau][s];
            tma_bulk_g2s(sA + buf * PP * PP, ops + (size_t)code * PP * PP, kOpBytes, &bar[buf]);
        }
        __syncthreads();  // expect_tx precedes the column copies
        if (tid < TN) {
            const int src = s_src[buf][tid];
            const float *gsrc = src >= 0 ? M + (size_t)src * PP : zero_block;
            fence_proxy_async();
            tma_bulk_g2s(sB + buf * TN * SB + tid * SB, gsrc, kColBytes, &bar[buf]);
        }
    };

    const int cg = tid % NCG, rg = tid / NCG;
    float acc[RM][CN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) acc[i][j] = 0.f;

    constexpr int S = 189;
    uint32_t phase[2] = {0u, 0u};
    resolve(0, 0);
    __syncthreads();
    issue(0, 0);
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        if (s + 1 < S) {
            resolve(s + 1, buf ^ 1);
            __syncthreads();  // s_src published; everyone finished reading buffer buf^1 (slot s-1)
            issue(s + 1, buf ^ 1);
        }
        if (mbar_wait_bounded(&bar[buf], phase[buf], kWaitLimitNs))
            phase[buf] ^= 1u;
        else
            s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        const float *A = sA + buf * PP * PP + rg * RM;
        const float *B = sB + buf * TN * SB + cg * SB;
#pragma unroll 2
        for (int k = 0; k < PP; k += 4) {
            float4 b[CN];
#pragma unroll
            for (int j = 0; j < CN; ++j) b[j] = *reinterpret_cast<const float4 *>(B + j * NCG * SB + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 a = *reinterpret_cast<const float4 *>(A + (k + kk) * PP);
#pragma unroll
                for (int j = 0; j < CN; ++j) {
                    const float bv = kk == 0 ? b[j].x : kk == 1 ? b[j].y : kk == 2 ? b[j].z : b[j].w;
                    acc[0][j] = fmaf(a.x, bv, acc[0][j]);
                    acc[1][j] = fmaf(a.y, bv, acc[1][j]);
                    acc[2][j] = fmaf(a.z, bv, acc[2][j]);
                    acc[3][j] = fmaf(a.w, bv, acc[3][j]);
                }
            }
        }
    }
    if (s_abort) {
        if (tid == 0) atomicOr(status, kStatusTimeout);
        // let copies in flight land before the CTA's shared memory is released (bounded)
        mbar_wait_bounded(&bar[0], phase[0], kWaitLimitNs);
        mbar_wait_bounded(&bar[1], phase[1], kWaitLimitNs);
        return;
    }
#pragma unroll
    for (int j = 0; j < CN; ++j) {
        const int t = cg + j * NCG;
        const int64_t q = q0 + t;
        if (q >= nq) continue;
        const int64_t g = off + 8 * q + tau;
        if (end[g] <= begin[g]) continue;
        float4 v = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        *reinterpret_cast<float4 *>(Lc + g * PP + rg * RM) = v;
    }
    (void)NTH;
}

template <int P, int TN, int RM, int CN>
static void launch_m2l_t(int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                         const int32_t *m2l_ids, const uint16_t *m2l_code, const float *ops, const float *M,
                         float *Lc, const float *zero_block, int *status, cudaStream_t s)
{
    constexpr int PP = P * P;
    constexpr int NTH = (PP / RM) * (TN / CN);
    const size_t smem = (size_t)(2 * PP * PP + 2 * TN * M2LShape<P>::SB) * sizeof(float);
    cudaFuncSetAttribute(k_m2l<P, TN, RM, CN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    M2LTiles tiles{};
    tiles.L = L;
    int total = 0;
    for (int l = 2; l <= L; ++l) {
        int64_t nq = int64_t(1) << (3 * (l - 1));
        tiles.ntiles_level[l] = (int)(8 * ((nq + TN - 1) / TN));
        total += tiles.ntiles_level[l];
    }
    if (total == 0) return;
    k_m2l<P, TN, RM, CN><<<total, NTH, smem, s>>>(tiles, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc,
                                                  zero_block, status);
    note_launches(1);
}

void launch_m2l(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                const int32_t *m2l_ids, const uint16_t *m2l_code, const float *ops, const float *M, float *Lc,
                const float *zero_block, int *status, cudaStream_t s)
{
    if (L < 2) return;
    switch (P) {
    case 4: launch_m2l_t<4, 32, 4, 4>(L, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    case 6: launch_m2l_t<6, 64, 4, 8>(L, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    case 8: launch_m2l_t<8, 64, 4, 8>(L, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    case 10: launch_m2l_t<10, 64, 4, 8>(L, begin, end, m2l_offs, m2l_ids, m2l_code, ops, M, Lc, zero_block, status, s); break;
    }
}

}  // namespace gbfmm
