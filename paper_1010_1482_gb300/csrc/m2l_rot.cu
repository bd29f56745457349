// M2L (Eq. 4) by rotation to the translation axis: O(p^3) work per (target, source) pair
// instead of the dense operator's O(p^4) (the rotation-based M2L of the FMM literature the
// paper cites in Section "Overview of Advanced Techniques").
//
// For the offset of a list entry the dense operator factors as T = F^-1 C F (factors from
// build_m2l_rot_table, checked there against the dense operator): F rotates the multipole
// expansion so that the translation runs along +z (a (2n+1) x (2n+1) block per degree n), C is
// the coaxial translation (a (p-m) x (p-m) block per order m, the same for the real and the
// imaginary parts), and F^-1 rotates the local expansion back.  Per pair at p = 10: 1330 + 770
// + 1330 multiply-adds against the dense 10,000.
//
// FP32 on the CUDA cores.  A CTA takes 64 targets of one level and one child position tau (they
// share the 189 admissible offsets) and walks the offsets in the lists' stencil-code order: the
// offset's three factors and the 64 targets' sources are staged in shared memory (sources
// transposed, one column per target), then the three stages run as small dense products, the
// last one accumulating each thread's (2 targets x 13 coefficients at p = 10) outputs in
// registers; each factor entry read from shared memory feeds both targets.
#include "common.cuh"

#include <vector>

namespace gbfmm {

size_t m2l_rot_code_floats(int P);
int build_m2l_rot_table(int P, std::vector<float> &out);

namespace {

constexpr int kRotTN = 64;        // targets per CTA
constexpr int kRotCol = kRotTN + 1;  // column stride of the staged vectors (bank-conflict free)
constexpr int kRotThreads = 256;

__constant__ uint16_t c_rot_codes[8][189];

template <int P>
struct RotCfg {
    static constexpr int PP = P * P;
    static constexpr int FSZ = P * (4 * P * P - 1) / 3;  // sum over n < P of (2n+1)^2
    static constexpr int CSZ = P * (P + 1) * (2 * P + 1) / 6;  // sum over m < P of (P-m)^2
    static constexpr int RS = (2 * FSZ + CSZ + 3) / 4 * 4;  // per code, 16-byte aligned
    static constexpr int RG = kRotThreads / (kRotTN / 2);  // row groups: 8 (each thread 2 targets)
    static constexpr int RPT = (PP + RG - 1) / RG;         // rows per thread
    static constexpr size_t kSmemBytes = ((size_t)RS + 3 * (size_t)PP * kRotCol) * sizeof(float);
};

struct RotTiles {
    int L;
    int ntiles_level[kMaxLevel + 1];
};

// per coefficient row r = (n, m, re/im): its F row (offset in the factor table), the first
// column of its degree block and the block's width, and its C row (offset) with the stride and
// the first column of its order
struct RotRow {
    short fofs, b, s, cofs, m, cb;
};

template <int P>
__global__ void __launch_bounds__(kRotThreads) k_m2l_rot(RotTiles tiles, const int32_t *__restrict__ begin,
                                                         const int32_t *__restrict__ end,
                                                         const uint32_t *__restrict__ m2l_offs,
                                                         const int32_t *__restrict__ m2l_ids,
                                                         const uint16_t *__restrict__ m2l_code,
                                                         const float *__restrict__ tab, const float *__restrict__ M,
                                                         float *__restrict__ Lc)
{
    using C = RotCfg<P>;
    constexpr int PP = C::PP, FSZ = C::FSZ, RS = C::RS, RG = C::RG, RPT = C::RPT;
    extern __shared__ __align__(16) float rot_smem[];
    float *sop = rot_smem;              // F | F^-1 | C of the current offset
    float *A = sop + RS;                // sources, [coefficient][target]
    float *W = A + PP * kRotCol;        // after F
    float *Z = W + PP * kRotCol;        // after C
    __shared__ uint32_t s_ptr[kRotTN], s_pend[kRotTN];
    __shared__ int s_src[kRotTN];
    __shared__ RotRow s_row[PP];

    // tile: levels L, L-1, ..., 2; in a level, child position tau, then blocks of 64 parents
    int rem = blockIdx.x, l = tiles.L;
    while (l >= 2 && rem >= tiles.ntiles_level[l]) rem -= tiles.ntiles_level[l--];
    if (l < 2) return;
    const int64_t nq = int64_t(1) << (3 * (l - 1));
    const int64_t qtiles = (nq + kRotTN - 1) / kRotTN;
    const int tau = (int)(rem / qtiles);
    const int64_t q0 = (rem % qtiles) * kRotTN, off = level_offset(l);
    const int tid = threadIdx.x;
    if (tid < kRotTN) {
        const int64_t q = q0 + tid;
        uint32_t p = 0, pe = 0;
        if (q < nq) {
            const int64_t g = off + 8 * q + tau;
            if (end[g] > begin[g]) {
                p = m2l_offs[g];
                pe = m2l_offs[g + 1];
            }
        }
        s_ptr[tid] = p;
        s_pend[tid] = pe;
    }
    for (int r = tid; r < PP; r += kRotThreads) {
        int n = 0;
        while ((n + 1) * (n + 1) <= r) ++n;
        const int b = n * n, sw = 2 * n + 1, rr = r - b;
        const int m = (rr + 1) / 2, im = rr > 0 && (rr % 2 == 0);
        int cofs = 2 * FSZ;
        for (int mm = 0; mm < m; ++mm) cofs += (P - mm) * (P - mm);
        cofs += (n - m) * (P - m);
        s_row[r] = RotRow{(short)((n * (4 * n * n - 1)) / 3 + rr * sw), (short)b, (short)sw, (short)cofs, (short)m,
                          (short)(m == 0 ? 0 : 2 * m - 1 + im)};
    }
    // thread: targets t and t + 32, coefficient rows rg, rg + RG, ...
    const int t = tid % 32, rg = tid / 32;
    float acc0[RPT], acc1[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc0[i] = acc1[i] = 0.f;
    __syncthreads();

    for (int k = 0; k < 189; ++k) {
        const int code = c_rot_codes[tau][k];
        // the offset's factors, each target's source of this offset (lists are in code order)
        const float4 *src_op = reinterpret_cast<const float4 *>(tab + (size_t)code * RS);
        for (int e = tid; e < RS / 4; e += kRotThreads) reinterpret_cast<float4 *>(sop)[e] = __ldg(&src_op[e]);
        if (tid < kRotTN) {
            int s = -1;
            const uint32_t p = s_ptr[tid];
            if (p < s_pend[tid] && m2l_code[p] == code) {
                s = m2l_ids[p];
                s_ptr[tid] = p + 1;
            }
            s_src[tid] = s;
        }
        __syncthreads();
        // gather, one warp per target at a time (coalesced rows), transposed into A
        for (int tt = tid >> 5; tt < kRotTN; tt += kRotThreads / 32) {
            const int s = s_src[tt];
            for (int j = tid & 31; j < PP; j += 32) A[j * kRotCol + tt] = s >= 0 ? __ldg(&M[(size_t)s * PP + j]) : 0.f;
        }
        __syncthreads();
        // W = F A (block-diagonal in the degree)
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = rg + RG * i;
            if (r >= PP) break;
            const RotRow w = s_row[r];
            const float *f = sop + w.fofs, *a = A + w.b * kRotCol + t;
            float v0 = 0.f, v1 = 0.f;
            for (int c = 0; c < w.s; ++c) {
                const float fc = f[c];
                v0 = fmaf(fc, a[c * kRotCol], v0);
                v1 = fmaf(fc, a[c * kRotCol + 32], v1);
            }
            W[r * kRotCol + t] = v0;
            W[r * kRotCol + t + 32] = v1;
        }
        __syncthreads();
        // Z = C W (order blocks: row (j, m, re/im) from columns (n, m, re/im), n = m .. P-1)
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = rg + RG * i;
            if (r >= PP) break;
            const RotRow w = s_row[r];
            const float *crow = sop + w.cofs;
            float v0 = 0.f, v1 = 0.f;
            for (int n = w.m; n < P; ++n) {
                const float cv = crow[n - w.m];
                const float *wc = W + (n * n + w.cb) * kRotCol + t;
                v0 = fmaf(cv, wc[0], v0);
                v1 = fmaf(cv, wc[32], v1);
            }
            Z[r * kRotCol + t] = v0;
            Z[r * kRotCol + t + 32] = v1;
        }
        __syncthreads();
        // L += F^-1 Z
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = rg + RG * i;
            if (r >= PP) break;
            const RotRow w = s_row[r];
            const float *f = sop + FSZ + w.fofs, *z = Z + w.b * kRotCol + t;
            float v0 = acc0[i], v1 = acc1[i];
            for (int c = 0; c < w.s; ++c) {
                const float fc = f[c];
                v0 = fmaf(fc, z[c * kRotCol], v0);
                v1 = fmaf(fc, z[c * kRotCol + 32], v1);
            }
            acc0[i] = v0;
            acc1[i] = v1;
        }
        __syncthreads();  // sop, A, W and Z are refilled for the next offset
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t q = q0 + t + 32 * h;
        if (q >= nq) continue;
        const int64_t g = off + 8 * q + tau;
        if (end[g] <= begin[g]) continue;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int r = rg + RG * i;
            if (r < PP) Lc[g * PP + r] = h ? acc1[i] : acc0[i];
        }
    }
}

template <int P>
void launch_rot_t(const RotTiles &tiles, int total, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                  const int32_t *m2l_ids, const uint16_t *m2l_code, const float *tab, const float *M, float *Lc,
                  cudaStream_t s)
{
    using C = RotCfg<P>;
    cudaFuncSetAttribute(k_m2l_rot<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmemBytes);
    k_m2l_rot<P><<<total, kRotThreads, C::kSmemBytes, s>>>(tiles, begin, end, m2l_offs, m2l_ids, m2l_code, tab, M, Lc);
    note_launches(1);
}

}  // namespace

void init_m2l_rot_constants()
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
    cudaMemcpyToSymbol(c_rot_codes, codes, sizeof(codes));
}

size_t m2l_rot_table_bytes(int P) { return m2l_rot_code_floats(P) * kM2LCodes * sizeof(float); }

// host FP64 factors (checked), copied to `table` (device); synchronous.  0 on success.
int build_m2l_rot(int P, void *table)
{
    std::vector<float> h;
    const int rc = build_m2l_rot_table(P, h);
    if (rc != 0) return rc;
    return cudaMemcpy(table, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? 0 : -10;
}

// M2L of levels 2..L of the uniform tree over its M2L lists (table: build_m2l_rot)
void launch_m2l_rot(int P, int L, const int32_t *begin, const int32_t *end, const uint32_t *m2l_offs,
                    const int32_t *m2l_ids, const uint16_t *m2l_code, const void *table, const float *M, float *Lc,
                    cudaStream_t s)
{
    if (L < 2) return;
    RotTiles tiles{};
    tiles.L = L;
    int total = 0;
    for (int l = 2; l <= L; ++l) {
        const int64_t nq = int64_t(1) << (3 * (l - 1));
        tiles.ntiles_level[l] = (int)(8 * ((nq + kRotTN - 1) / kRotTN));
        total += tiles.ntiles_level[l];
    }
    const float *tab = static_cast<const float *>(table);
    switch (P) {
    case 4: launch_rot_t<4>(tiles, total, begin, end, m2l_offs, m2l_ids, m2l_code, tab, M, Lc, s); break;
    case 6: launch_rot_t<6>(tiles, total, begin, end, m2l_offs, m2l_ids, m2l_code, tab, M, Lc, s); break;
    case 8: launch_rot_t<8>(tiles, total, begin, end, m2l_offs, m2l_ids, m2l_code, tab, M, Lc, s); break;
    case 10: launch_rot_t<10>(tiles, total, begin, end, m2l_offs, m2l_ids, m2l_code, tab, M, Lc, s); break;
    }
}

}  // namespace gbfmm
