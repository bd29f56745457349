// P2P near field (Section "The P2P kernel implementation", Listings 1-2) and the direct
// all-pairs sum (Eq. 1), FP32 with the reciprocal square root.
//
// Pair rule (both kernels): with d = x_i - x_j and d2 = |d|^2,
//   phi_i  += q_j / sqrt(d2 + eps2),   grad_i -= q_j d / (d2 + eps2)^(3/2),
// and pairs with d2 == 0 (the particle itself, exact duplicates) contribute nothing.
//
// Decomposition: one CTA (128 threads) per target leaf.  The leaf's neighbour cells (the
// uniform tree's <= 27, or an adaptive leaf's U list) are gathered into shared memory in chunks,
// as packed pairs (x, x | y, y), (z, z | q, q).  Each thread holds two targets in one 64-bit
// register per coordinate and applies the pair rule with packed FP32x2 instructions, so one
// staged source feeds two pair interactions; when the leaf has fewer target slots than the CTA
// has threads, the threads form G groups that split the sources round-robin, so the lanes stay
// busy for leaves of any occupancy (the paper instead pads targets to the block size).  Each
// thread sums its share in FP32; the group partials are combined per target with compensated
// (Kahan) summation.  Then either the far-field value is added the same way and the result
// written to the caller's original particle order, or (FMM) the compensated sums are stored for
// L2P, which adds the far field and writes the output.
#include "common.cuh"

namespace gbfmm {

constexpr int kP2PThreads = 128;
constexpr int kRowCap = 32;

template <bool SOFT>
GB_DEV void pair(float xi, float yi, float zi, float4 s, float eps2, float &phi, float &gx, float &gy, float &gz)
{
    const float dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrt_ftz(SOFT ? d2 + eps2 : d2);
    inv = d2 > 0.f ? inv : 0.f;
    const float qi = s.w * inv;
    phi += qi;
    const float qi3 = qi * inv * inv;
    gx = fmaf(-dx, qi3, gx);
    gy = fmaf(-dy, qi3, gy);
    gz = fmaf(-dz, qi3, gz);
}

// ---- packed FP32x2 arithmetic (two lanes of one 64-bit register: targets a and b) -------------
GB_DEV uint64_t f2_pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
GB_DEV void f2_unpack(uint64_t r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
GB_DEV uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
GB_DEV uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
GB_DEV uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
GB_DEV uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The pair rule for two targets at once (packed X, Y, Z) and one source whose coordinates and
// charge are staged duplicated: xy = (x, x, y, y), zq = (z, z, q, q).  Same operation order as
// pair(); the gradient accumulates +d q / r^3 and is negated once at the end.  MASK drops pairs
// at zero distance (only the target's own cell can hold them).
template <bool SOFT, bool MASK>
GB_DEV void pair2(uint64_t X, uint64_t Y, uint64_t Z, ulonglong2 xy, ulonglong2 zq, uint64_t E2, uint64_t &P,
                  uint64_t &GX, uint64_t &GY, uint64_t &GZ)
{
    const uint64_t dx = f2_sub(X, xy.x);
    const uint64_t dy = f2_sub(Y, xy.y);
    const uint64_t dz = f2_sub(Z, zq.x);
    uint64_t d2 = f2_mul(dz, dz);
    d2 = f2_fma(dy, dy, d2);
    d2 = f2_fma(dx, dx, d2);
    float r0, r1;
    f2_unpack(SOFT ? f2_add(d2, E2) : d2, r0, r1);
    float i0 = rsqrt_ftz(r0), i1 = rsqrt_ftz(r1);
    if (MASK) {
        float a0, a1;
        f2_unpack(d2, a0, a1);
        i0 = a0 > 0.f ? i0 : 0.f;
        i1 = a1 > 0.f ? i1 : 0.f;
    }
    const uint64_t inv = f2_pack(i0, i1);
    const uint64_t w = f2_mul(zq.y, inv);
    P = f2_add(P, w);
    const uint64_t w3 = f2_mul(f2_mul(w, inv), inv);
    GX = f2_fma(dx, w3, GX);
    GY = f2_fma(dy, w3, GY);
    GZ = f2_fma(dz, w3, GZ);
}

constexpr int kSrcCap2 = 512;

// CTA per target leaf, TPT targets per thread in packed pairs; the leaf's own cell is staged
// first so that only its sources pay for the zero-distance test
template <bool SOFT, int TPT, int NT = kP2PThreads>
__global__ void __launch_bounds__(NT) k_p2p2(int L, const int32_t *__restrict__ leaves,
                                                      const float4 *__restrict__ sx,
                                                      const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
                                                      const uint32_t *__restrict__ p2p_offs,
                                                      const int32_t *__restrict__ p2p_ids,
                                                      const float4 *__restrict__ far,
                                                      const uint32_t *__restrict__ perm, float eps2,
                                                      float4 *__restrict__ out, float4 *__restrict__ near, Span lv)
{
    constexpr int NPK = TPT / 2;
    if (leaves && blockIdx.x >= span_count(lv)) return;  // beyond the listed leaves
    __shared__ ulonglong2 sA[kSrcCap2], sB[kSrcCap2];  // (x, x | y, y), (z, z | q, q)
    __shared__ float4 red[TPT][NT];
    __shared__ int s_cb[kRowCap], s_pref[kRowCap + 1], s_self;
    const int64_t leaf = leaves ? (int64_t)leaves[blockIdx.x] : (int64_t)blockIdx.x;
    const int64_t g = leaves ? leaf : level_offset(L) + leaf;
    const int b0 = begin[g], e0 = end[g];
    if (e0 <= b0) return;
    const int tid = threadIdx.x;
    const uint32_t r0 = p2p_offs[leaf];
    const int nrow = (int)(p2p_offs[leaf + 1] - r0);
    const int T = e0 - b0;
    const uint64_t E2 = f2_pack(eps2, eps2);
    for (int tc = 0; tc < T; tc += TPT * NT) {
        const int Tc = min(T - tc, TPT * NT);
        const int slots = (Tc + TPT - 1) / TPT;
        const int G = NT / slots;
        const int slot = tid % slots, grp = tid / slots;
        const bool active = grp < G;
        uint64_t X[NPK], Y[NPK], Z[NPK], P[NPK], GX[NPK], GY[NPK], GZ[NPK];
#pragma unroll
        for (int k = 0; k < NPK; ++k) {
            // a missing target repeats the slot's first one; its result is discarded
            const int ta = TPT * slot + 2 * k, tb = ta + 1;
            const float4 pa = __ldg(&sx[b0 + tc + (ta < Tc ? ta : TPT * slot)]);
            const float4 pb = __ldg(&sx[b0 + tc + (tb < Tc ? tb : TPT * slot)]);
            X[k] = f2_pack(pa.x, pb.x);
            Y[k] = f2_pack(pa.y, pb.y);
            Z[k] = f2_pack(pa.z, pb.z);
            P[k] = GX[k] = GY[k] = GZ[k] = 0ull;
        }
        for (int rb = 0; rb < nrow; rb += kRowCap) {
            const int nr = min(kRowCap, nrow - rb);
            __syncthreads();
            if (tid < nr) {
                const int c = p2p_ids[r0 + rb + tid];
                s_cb[tid] = begin[c];
                s_pref[tid + 1] = end[c] - begin[c];
            }
            __syncthreads();
            if (tid == 0) {
                // the target's own cell first
                int self = 0;
                for (int k = 0; k < nr; ++k)
                    if (s_cb[k] == b0 && s_pref[k + 1] == T) {
                        const int cb = s_cb[k], cn = s_pref[k + 1];
                        s_cb[k] = s_cb[0];
                        s_pref[k + 1] = s_pref[1];
                        s_cb[0] = cb;
                        s_pref[1] = cn;
                        self = T;
                        break;
                    }
                s_self = self;
                s_pref[0] = 0;
                for (int k = 0; k < nr; ++k) s_pref[k + 1] += s_pref[k];
            }
            __syncthreads();
            const int S = s_pref[nr], nself = s_self;
            for (int sc = 0; sc < S; sc += kSrcCap2) {
                const int chunk = min(kSrcCap2, S - sc);
                if (sc > 0) __syncthreads();
                // warp w stages rows w, w + 4, ... (its lanes stride the row's particles)
                for (int e = tid >> 5; e < nr; e += NT / 32) {
                    const int lo = max(s_pref[e], sc), hi = min(s_pref[e + 1], sc + chunk);
                    for (int q = lo + (tid & 31); q < hi; q += 32) {
                        const float4 p = __ldg(&sx[s_cb[e] + (q - s_pref[e])]);
                        sA[q - sc] = make_ulonglong2(f2_pack(p.x, p.x), f2_pack(p.y, p.y));
                        sB[q - sc] = make_ulonglong2(f2_pack(p.z, p.z), f2_pack(p.w, p.w));
                    }
                }
                __syncthreads();
                if (active) {
                    const int mend = max(0, min(chunk, nself - sc));
                    int j = grp;
                    for (; j < mend; j += G) {
                        const ulonglong2 a = sA[j], b = sB[j];
#pragma unroll
                        for (int k = 0; k < NPK; ++k) pair2<SOFT, true>(X[k], Y[k], Z[k], a, b, E2, P[k], GX[k], GY[k], GZ[k]);
                    }
#pragma unroll 4
                    for (; j < chunk; j += G) {
                        const ulonglong2 a = sA[j], b = sB[j];
#pragma unroll
                        for (int k = 0; k < NPK; ++k) pair2<SOFT, false>(X[k], Y[k], Z[k], a, b, E2, P[k], GX[k], GY[k], GZ[k]);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NPK; ++k) {
            float p0, p1, x0, x1, y0, y1, z0, z1;
            f2_unpack(P[k], p0, p1);
            f2_unpack(GX[k], x0, x1);
            f2_unpack(GY[k], y0, y1);
            f2_unpack(GZ[k], z0, z1);
            red[2 * k][tid] = make_float4(p0, -x0, -y0, -z0);
            red[2 * k + 1][tid] = make_float4(p1, -x1, -y1, -z1);
        }
        __syncthreads();
        if (grp == 0) {
#pragma unroll
            for (int h = 0; h < TPT; ++h) {
                const int t = TPT * slot + h;
                if (t >= Tc) break;
                const int i = b0 + tc + t;
                Kahan a{0.f, 0.f}, bx{0.f, 0.f}, by{0.f, 0.f}, bz{0.f, 0.f};
                for (int k = 0; k < G; ++k) {
                    const float4 v = red[h][k * slots + slot];
                    a.add(v.x);
                    bx.add(v.y);
                    by.add(v.z);
                    bz.add(v.w);
                }
                if (near) {  // the compensated sums so far; the far field is added by L2P
                    near[2 * (int64_t)i] = make_float4(a.s, bx.s, by.s, bz.s);
                    near[2 * (int64_t)i + 1] = make_float4(a.c, bx.c, by.c, bz.c);
                    continue;
                }
                if (far) {
                    const float4 f = far[i];
                    a.add(f.x);
                    bx.add(f.y);
                    by.add(f.z);
                    bz.add(f.w);
                }
                out[perm[i]] = make_float4(a.s, bx.s, by.s, bz.s);
            }
        }
    }
}

// ---- launchers --------------------------------------------------------------------------------
// the largest shared-memory carveout, so that the kernel's CTAs can share an SM with a tensor-core
// M2L's when both run at once
static void launch_leaf(unsigned grid, int L, const int32_t *leaves, const float4 *sx, const int32_t *begin,
                        const int32_t *end, const uint32_t *offs, const int32_t *ids, const float4 *far,
                        const uint32_t *perm, float eps2, float4 *out, float4 *near, cudaStream_t s,
                        Span lv = Span{})
{
    static const bool carve = [] {
        cudaFuncSetAttribute(k_p2p2<true, 2, kP2PThreads>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_p2p2<false, 2, kP2PThreads>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        return true;
    }();
    (void)carve;
    if (eps2 > 0.f)
        k_p2p2<true, 2, kP2PThreads><<<grid, kP2PThreads, 0, s>>>(L, leaves, sx, begin, end, offs, ids, far, perm,
                                                                  eps2, out, near, lv);
    else
        k_p2p2<false, 2, kP2PThreads><<<grid, kP2PThreads, 0, s>>>(L, leaves, sx, begin, end, offs, ids, far, perm,
                                                                   eps2, out, near, lv);
    note_launches(1);
}

void launch_p2p(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs,
                const int32_t *p2p_ids, const float4 *far, const uint32_t *perm, float eps2, float4 *out,
                cudaStream_t s)
{
    if (n <= 0) return;
    launch_leaf((unsigned)(int64_t(1) << (3 * L)), L, nullptr, sx, begin, end, p2p_offs, p2p_ids, far, perm, eps2,
                out, nullptr, s);
}

void launch_p2p_cells(const int32_t *leaves, Span lv, int64_t n, const float4 *sx, const int32_t *begin,
                      const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, const float4 *far,
                      const uint32_t *perm, float eps2, float4 *out, cudaStream_t s)
{
    if (n <= 0 || lv.cap <= 0) return;
    launch_leaf((unsigned)lv.cap, 0, leaves, sx, begin, end, u_offs, u_ids, far, perm, eps2, out, nullptr, s, lv);
}

bool p2p_near_supported() { return true; }

void launch_p2p_near(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end,
                     const uint32_t *p2p_offs, const int32_t *p2p_ids, float eps2, float4 *near, cudaStream_t s)
{
    if (n <= 0) return;
    launch_leaf((unsigned)(int64_t(1) << (3 * L)), L, nullptr, sx, begin, end, p2p_offs, p2p_ids, nullptr, nullptr,
                eps2, nullptr, near, s);
}

void launch_p2p_cells_near(const int32_t *leaves, Span lv, int64_t n, const float4 *sx, const int32_t *begin,
                           const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, float eps2, float4 *near,
                           cudaStream_t s)
{
    if (n <= 0 || lv.cap <= 0) return;
    launch_leaf((unsigned)lv.cap, 0, leaves, sx, begin, end, u_offs, u_ids, nullptr, nullptr, eps2, nullptr, near, s,
                lv);
}

// Direct all-pairs sum: one thread per target, sources streamed through shared memory in
// tiles of the block size (the tile model of the GPU Gems 3 all-pairs kernel the paper builds on).
constexpr int kDirectThreads = 256;

template <bool SOFT>
__global__ void __launch_bounds__(kDirectThreads) k_direct(int64_t ns, const float4 *__restrict__ src, int64_t nt,
                                                           const float4 *__restrict__ tgt, float eps2,
                                                           float4 *__restrict__ out)
{
    __shared__ float4 tile[kDirectThreads];
    const int64_t i = blockIdx.x * (int64_t)kDirectThreads + threadIdx.x;
    const float4 xi = i < nt ? __ldg(&tgt[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    float phi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    for (int64_t b = 0; b < ns; b += kDirectThreads) {
        const int64_t j = b + threadIdx.x;
        tile[threadIdx.x] = j < ns ? __ldg(&src[j]) : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int cnt = (int)(ns - b < kDirectThreads ? ns - b : kDirectThreads);
#pragma unroll 8
        for (int k = 0; k < cnt; ++k) pair<SOFT>(xi.x, xi.y, xi.z, tile[k], eps2, phi, gx, gy, gz);
        __syncthreads();
    }
    if (i < nt) out[i] = make_float4(phi, gx, gy, gz);
}

void launch_direct(int64_t n_src, const float4 *src, int64_t n_tgt, const float4 *tgt, float eps2, float4 *out,
                   cudaStream_t s)
{
    if (n_tgt <= 0) return;
    unsigned grid = (unsigned)((n_tgt + kDirectThreads - 1) / kDirectThreads);
    if (eps2 > 0.f)
        k_direct<true><<<grid, kDirectThreads, 0, s>>>(n_src, src, n_tgt, tgt, eps2, out);
    else
        k_direct<false><<<grid, kDirectThreads, 0, s>>>(n_src, src, n_tgt, tgt, eps2, out);
    note_launches(1);
}

}  // namespace gbfmm
