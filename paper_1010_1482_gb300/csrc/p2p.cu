// P2P near field (Section "The P2P kernel implementation", Listings 1-2) and the direct
// all-pairs sum (Eq. 1), FP32 with the reciprocal square root.
//
// Pair rule (both kernels): with d = x_i - x_j and d2 = |d|^2,
//   phi_i  += q_j / sqrt(d2 + eps2),   grad_i -= q_j d / (d2 + eps2)^(3/2),
// and pairs with d2 == 0 (the particle itself, exact duplicates) contribute nothing.
//
// Decomposition: one CTA per target leaf.  The leaf's <= 27 neighbour cells are gathered into
// shared memory (float4 x, y, z, q, in chunks).  Each thread holds TPT targets in registers,
// so one staged source feeds TPT pair interactions; when the leaf has fewer target slots than
// the CTA has threads, the threads form G groups that split the sources round-robin, so the
// lanes stay busy for leaves of any occupancy (the paper instead pads targets to the block
// size).  Each thread sums its share in FP32; the group partials are combined per target with
// compensated (Kahan) summation.  Then either the far-field value is added the same way and the
// result written to the caller's original particle order, or (FMM, the packed-pair kernels) the
// compensated sums are stored for L2P, which adds the far field and writes the output.
#include "common.cuh"

#include <stdlib.h>

namespace gbfmm {

constexpr int kP2PThreads = 128;

// P2P kernel (GBFMM_P2P_TPT): 12 / 14 = CTA per leaf, packed FP32x2 pairs, 2 / 4 targets per
// thread (12 is the default); 16 / 17 = as 12 with 64 / 256 threads per CTA; 0 = warp per leaf;
// 1, 2, 4, 8 = CTA per leaf, scalar FP32, that many targets per thread
static int p2p_tpt()
{
    static const int v = [] {
        const char *e = getenv("GBFMM_P2P_TPT");
        const int x = e ? atoi(e) : 12;
        return (x == 0 || x == 1 || x == 2 || x == 4 || x == 8 || x == 12 || x == 14 || x == 16 || x == 17 ||
                x == 20)
                   ? x
                   : 12;
    }();
    return v;
}
constexpr int kSrcCap = 1024;
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

template <bool SOFT, int TPT>
__global__ void __launch_bounds__(kP2PThreads) k_p2p(int L, const int32_t *__restrict__ leaves,
                                                     const float4 *__restrict__ sx,
                                                     const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
                                                     const uint32_t *__restrict__ p2p_offs,
                                                     const int32_t *__restrict__ p2p_ids, const float4 *__restrict__ far,
                                                     const uint32_t *__restrict__ perm, float eps2,
                                                     float4 *__restrict__ out)
{
    __shared__ float4 src[kSrcCap];
    __shared__ float4 red[TPT][kP2PThreads];
    __shared__ int s_cb[kRowCap], s_pref[kRowCap + 1];
    // target leaf: dense leaf blockIdx.x of a uniform depth-L tree (list row = leaf), or the
    // listed cell of an adaptive tree (list row = cell index)
    const int64_t leaf = leaves ? (int64_t)leaves[blockIdx.x] : (int64_t)blockIdx.x;
    const int64_t g = leaves ? leaf : level_offset(L) + leaf;
    const int b0 = begin[g], e0 = end[g];
    if (e0 <= b0) return;
    const int tid = threadIdx.x;
    const uint32_t r0 = p2p_offs[leaf];
    const int nrow = (int)(p2p_offs[leaf + 1] - r0);
    const int T = e0 - b0;
    for (int tc = 0; tc < T; tc += TPT * kP2PThreads) {
        const int Tc = min(T - tc, TPT * kP2PThreads);
        const int slots = (Tc + TPT - 1) / TPT;
        const int G = kP2PThreads / slots;
        const int slot = tid % slots, grp = tid / slots;
        const bool active = grp < G;
        float tx[TPT], ty[TPT], tz[TPT];
        float phi[TPT], gx[TPT], gy[TPT], gz[TPT];
#pragma unroll
        for (int h = 0; h < TPT; ++h) {
            // a missing target repeats the slot's first one; its result is discarded
            const int t = TPT * slot + h < Tc ? TPT * slot + h : TPT * slot;
            const float4 p = __ldg(&sx[b0 + tc + t]);
            tx[h] = p.x;
            ty[h] = p.y;
            tz[h] = p.z;
            phi[h] = gx[h] = gy[h] = gz[h] = 0.f;
        }
        // source cells in blocks of kRowCap list entries (a uniform tree has <= 27; an
        // adaptive leaf may touch more, smaller leaves)
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
                s_pref[0] = 0;
                for (int k = 0; k < nr; ++k) s_pref[k + 1] += s_pref[k];
            }
            __syncthreads();
            const int S = s_pref[nr];
            for (int sc = 0; sc < S; sc += kSrcCap) {
                const int chunk = min(kSrcCap, S - sc);
                if (sc > 0) __syncthreads();
                for (int k = tid; k < chunk; k += kP2PThreads) {
                    const int s = sc + k;
                    int e = 0;
                    while (s >= s_pref[e + 1]) ++e;
                    src[k] = __ldg(&sx[s_cb[e] + (s - s_pref[e])]);
                }
                __syncthreads();
                if (active) {
#pragma unroll 4
                    for (int j = grp; j < chunk; j += G) {
                        const float4 s = src[j];
#pragma unroll
                        for (int h = 0; h < TPT; ++h)
                            pair<SOFT>(tx[h], ty[h], tz[h], s, eps2, phi[h], gx[h], gy[h], gz[h]);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < TPT; ++h) red[h][tid] = make_float4(phi[h], gx[h], gy[h], gz[h]);
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

// CTA per target leaf with TPT (2 or 4) targets per thread in packed pairs; the leaf's own cell
// is staged first so that only its sources pay for the zero-distance test
template <bool SOFT, int TPT, int NT = kP2PThreads>
__global__ void __launch_bounds__(NT) k_p2p2(int L, const int32_t *__restrict__ leaves,
                                                      const float4 *__restrict__ sx,
                                                      const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
                                                      const uint32_t *__restrict__ p2p_offs,
                                                      const int32_t *__restrict__ p2p_ids,
                                                      const float4 *__restrict__ far,
                                                      const uint32_t *__restrict__ perm, float eps2,
                                                      float4 *__restrict__ out, float4 *__restrict__ near)
{
    constexpr int NPK = TPT / 2;
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

// Uniform tree, CTA per parent cell ("superleaf"): the 4 x 4 x 4 leaves around the parent's 8
// children hold every source any child needs; they are staged once in shared memory (float4,
// cell by cell), then each thread takes two targets of one child (a packed pair) and sweeps the
// child's 27 neighbour cells from shared memory.  No per-leaf setup, no group split and no
// cross-thread reduction.  A block whose 64 cells hold more than kSuperCap particles sweeps
// the same cells from global memory instead.
constexpr int kSuperThreads = 128;
constexpr int kSuperCap = 2304;

template <bool SOFT, bool STAGED>
GB_DEV void super_sweep(const float4 *__restrict__ src, const int *cbeg, const int *ccnt, int lc, uint64_t X, uint64_t Y,
                        uint64_t Z, uint64_t E2, uint64_t &P, uint64_t &GX, uint64_t &GY, uint64_t &GZ)
{
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int cell = lc + dx + 4 * dy + 16 * dz;
                const int b = cbeg[cell], n = ccnt[cell];
                if (dx == 0 && dy == 0 && dz == 0) {
                    for (int j = 0; j < n; ++j) {
                        const float4 q = STAGED ? src[b + j] : __ldg(&src[b + j]);
                        pair2<SOFT, true>(X, Y, Z, make_ulonglong2(f2_pack(q.x, q.x), f2_pack(q.y, q.y)),
                                          make_ulonglong2(f2_pack(q.z, q.z), f2_pack(q.w, q.w)), E2, P, GX, GY, GZ);
                    }
                } else {
#pragma unroll 4
                    for (int j = 0; j < n; ++j) {
                        const float4 q = STAGED ? src[b + j] : __ldg(&src[b + j]);
                        pair2<SOFT, false>(X, Y, Z, make_ulonglong2(f2_pack(q.x, q.x), f2_pack(q.y, q.y)),
                                           make_ulonglong2(f2_pack(q.z, q.z), f2_pack(q.w, q.w)), E2, P, GX, GY, GZ);
                    }
                }
            }
}

template <bool SOFT>
__global__ void __launch_bounds__(kSuperThreads) k_p2p_super(int L, const float4 *__restrict__ sx,
                                                              const int32_t *__restrict__ begin,
                                                              const int32_t *__restrict__ end,
                                                              const float4 *__restrict__ far,
                                                              const uint32_t *__restrict__ perm, float eps2,
                                                              float4 *__restrict__ out)
{
    __shared__ float4 stage[kSuperCap];
    __shared__ int s_gbeg[64], s_cnt[64], s_beg[64], s_pp[9];
    __shared__ int s_total;
    const int tid = threadIdx.x;
    const int side = 1 << L;
    int px, py, pz;
    demorton3((uint32_t)blockIdx.x, px, py, pz);
    const int64_t loff = level_offset(L);
    if (tid < 64) {
        const int x = 2 * px - 1 + (tid & 3), y = 2 * py - 1 + ((tid >> 2) & 3), z = 2 * pz - 1 + (tid >> 4);
        int gb = 0, n = 0;
        if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
            const int64_t gi = loff + morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
            gb = begin[gi];
            n = end[gi] - gb;
            if (n < 0) n = 0;
        }
        s_gbeg[tid] = gb;
        s_cnt[tid] = n;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int c = 0; c < 64; ++c) {
            s_beg[c] = acc;
            acc += s_cnt[c];
        }
        s_total = acc;
        // target pairs of the 8 children (local cells (1 + (c & 1), 1 + ((c >> 1) & 1), 1 + (c >> 2)))
        s_pp[0] = 0;
        for (int c = 0; c < 8; ++c) {
            const int lc = (1 + (c & 1)) + 4 * (1 + ((c >> 1) & 1)) + 16 * (1 + (c >> 2));
            s_pp[c + 1] = s_pp[c] + (s_cnt[lc] + 1) / 2;
        }
    }
    __syncthreads();
    const bool staged = s_total <= kSuperCap;
    if (staged) {
        const int w = tid >> 5, lane = tid & 31;
        for (int c = w; c < 64; c += kSuperThreads / 32) {
            const int gb = s_gbeg[c], n = s_cnt[c], sb = s_beg[c];
            for (int j = lane; j < n; j += 32) stage[sb + j] = __ldg(&sx[gb + j]);
        }
        __syncthreads();
    }
    const uint64_t E2 = f2_pack(eps2, eps2);
    const int npairs = s_pp[8];
    for (int pi = tid; pi < npairs; pi += kSuperThreads) {
        int c = 0;
        while (pi >= s_pp[c + 1]) ++c;
        const int lc = (1 + (c & 1)) + 4 * (1 + ((c >> 1) & 1)) + 16 * (1 + (c >> 2));
        const int n = s_cnt[lc];
        const int ka = 2 * (pi - s_pp[c]), kb = ka + 1 < n ? ka + 1 : ka;
        const int ga = s_gbeg[lc] + ka, gbi = s_gbeg[lc] + kb;
        const float4 ta = __ldg(&sx[ga]), tb = __ldg(&sx[gbi]);
        const uint64_t X = f2_pack(ta.x, tb.x), Y = f2_pack(ta.y, tb.y), Z = f2_pack(ta.z, tb.z);
        uint64_t P = 0ull, GX = 0ull, GY = 0ull, GZ = 0ull;
        if (staged)
            super_sweep<SOFT, true>(stage, s_beg, s_cnt, lc, X, Y, Z, E2, P, GX, GY, GZ);
        else
            super_sweep<SOFT, false>(sx, s_gbeg, s_cnt, lc, X, Y, Z, E2, P, GX, GY, GZ);
        float p0, p1, x0, x1, y0, y1, z0, z1;
        f2_unpack(P, p0, p1);
        f2_unpack(GX, x0, x1);
        f2_unpack(GY, y0, y1);
        f2_unpack(GZ, z0, z1);
        {
            const float4 f = far ? far[ga] : make_float4(0.f, 0.f, 0.f, 0.f);
            out[perm[ga]] = make_float4(p0 + f.x, f.y - x0, f.z - y0, f.w - z0);
        }
        if (kb != ka) {
            const float4 f = far ? far[gbi] : make_float4(0.f, 0.f, 0.f, 0.f);
            out[perm[gbi]] = make_float4(p1 + f.x, f.y - x1, f.z - y1, f.w - z1);
        }
    }
}

// Warp-per-leaf variant: each warp takes one target leaf (lane = target; a second target per
// lane for leaves of 33..64 targets, further blocks of 64 in turn) and streams the sources of
// the leaf's list through its own shared-memory buffer: the cells of the list are appended with
// coalesced float4 loads, 32 particles at a time, and each full buffer is swept by every lane.
// No block-wide barrier and no cross-thread reduction; each target's FP32 sum runs over the
// sources in list order, then the far-field value is added.
constexpr int kP2PWarps = 4;
constexpr int kP2PChunk = 256;  // sources per warp buffer (4 KB)

template <bool SOFT>
__global__ void __launch_bounds__(32 * kP2PWarps) k_p2p_warp(int L, int64_t nleaves, const int32_t *__restrict__ leaves,
                                                              const float4 *__restrict__ sx,
                                                              const int32_t *__restrict__ begin,
                                                              const int32_t *__restrict__ end,
                                                              const uint32_t *__restrict__ p2p_offs,
                                                              const int32_t *__restrict__ p2p_ids,
                                                              const float4 *__restrict__ far,
                                                              const uint32_t *__restrict__ perm, float eps2,
                                                              float4 *__restrict__ out)
{
    __shared__ float4 sbuf[kP2PWarps][kP2PChunk];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t li = (int64_t)blockIdx.x * kP2PWarps + w;
    if (li >= nleaves) return;
    const int64_t leaf = leaves ? (int64_t)leaves[li] : li;
    const int64_t g = leaves ? leaf : level_offset(L) + leaf;
    const int b0 = begin[g], e0 = end[g];
    if (e0 <= b0) return;
    const uint32_t r0 = p2p_offs[leaf], r1 = p2p_offs[leaf + 1];
    float4 *sb = sbuf[w];
    for (int t0 = b0; t0 < e0; t0 += 64) {
        const int ta = t0 + lane, tb = t0 + 32 + lane;
        const bool two = e0 - t0 > 32;  // warp-uniform
        const float4 pa = __ldg(&sx[ta < e0 ? ta : b0]);
        const float4 pb = __ldg(&sx[tb < e0 ? tb : b0]);
        float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f, bx = 0.f, by = 0.f, bz = 0.f, bw = 0.f;
        auto sweep = [&](int nsrc) {
            if (two) {
#pragma unroll 4
                for (int j = 0; j < nsrc; ++j) {
                    const float4 q = sb[j];
                    pair<SOFT>(pa.x, pa.y, pa.z, q, eps2, aw, ax, ay, az);
                    pair<SOFT>(pb.x, pb.y, pb.z, q, eps2, bw, bx, by, bz);
                }
            } else {
#pragma unroll 8
                for (int j = 0; j < nsrc; ++j) pair<SOFT>(pa.x, pa.y, pa.z, sb[j], eps2, aw, ax, ay, az);
            }
        };
        int fill = 0;
        for (uint32_t e = r0; e < r1; ++e) {
            const int c = p2p_ids[e];
            const int cb = begin[c], cn = end[c] - cb;
            for (int j0 = 0; j0 < cn; j0 += 32) {
                if (fill > kP2PChunk - 32) {
                    __syncwarp();
                    sweep(fill);
                    __syncwarp();
                    fill = 0;
                }
                const int m = min(32, cn - j0);
                if (lane < m) sb[fill + lane] = __ldg(&sx[cb + j0 + lane]);
                fill += m;
            }
        }
        __syncwarp();
        sweep(fill);
        __syncwarp();
        if (ta < e0) {
            float4 f = far ? far[ta] : make_float4(0.f, 0.f, 0.f, 0.f);
            out[perm[ta]] = make_float4(aw + f.x, ax + f.y, ay + f.z, az + f.w);
        }
        if (two && tb < e0) {
            float4 f = far ? far[tb] : make_float4(0.f, 0.f, 0.f, 0.f);
            out[perm[tb]] = make_float4(bw + f.x, bx + f.y, by + f.z, bz + f.w);
        }
    }
}

template <int TPT>
static void launch_p2p_t(unsigned grid, int L, const int32_t *leaves, const float4 *sx, const int32_t *begin,
                         const int32_t *end, const uint32_t *offs, const int32_t *ids, const float4 *far,
                         const uint32_t *perm, float eps2, float4 *out, cudaStream_t s)
{
    if (eps2 > 0.f)
        k_p2p<true, TPT><<<grid, kP2PThreads, 0, s>>>(L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out);
    else
        k_p2p<false, TPT><<<grid, kP2PThreads, 0, s>>>(L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out);
    note_launches(1);
}

// near != nullptr: write the compensated near-field sums (sorted order, 2 float4 per particle:
// the sums, then their compensations) instead of adding `far` and scattering to `out`; only the
// packed-pair kernels have this output (p2p_has_near)
static bool p2p_has_near()
{
    const int t = p2p_tpt();
    return t == 12 || t == 14 || t == 16 || t == 17;
}

// the packed-pair kernel, with the shared-memory carveout of the tensor-core M2L (the largest)
// so that its CTAs can share an SM with the M2L's when both run at once
template <int TPT, int NT>
static void launch_pk(bool soft, unsigned grid, int L, const int32_t *leaves, const float4 *sx, const int32_t *begin,
                      const int32_t *end, const uint32_t *offs, const int32_t *ids, const float4 *far,
                      const uint32_t *perm, float eps2, float4 *out, float4 *near, cudaStream_t s)
{
    static const bool carve = [] {
        cudaFuncSetAttribute(k_p2p2<true, TPT, NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_p2p2<false, TPT, NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        return true;
    }();
    (void)carve;
    if (soft)
        k_p2p2<true, TPT, NT><<<grid, NT, 0, s>>>(L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near);
    else
        k_p2p2<false, TPT, NT><<<grid, NT, 0, s>>>(L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near);
    note_launches(1);
}

static void dispatch_p2p(unsigned grid, int L, const int32_t *leaves, const float4 *sx, const int32_t *begin,
                         const int32_t *end, const uint32_t *offs, const int32_t *ids, const float4 *far,
                         const uint32_t *perm, float eps2, float4 *out, cudaStream_t s, float4 *near = nullptr)
{
    if (p2p_has_near()) {  // packed pairs: 12 / 14 = 2 / 4 targets per thread; 16 / 17 = 64 / 256 threads
        const int t = p2p_tpt();
        if (t == 12) launch_pk<2, kP2PThreads>(eps2 > 0.f, grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near, s);
        if (t == 14) launch_pk<4, kP2PThreads>(eps2 > 0.f, grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near, s);
        if (t == 16) launch_pk<2, 64>(eps2 > 0.f, grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near, s);
        if (t == 17) launch_pk<2, 256>(eps2 > 0.f, grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near, s);
        return;
    }
    if (p2p_tpt() == 20) {  // superleaf (uniform tree only) takes 12 for leaf lists
        launch_pk<2, kP2PThreads>(eps2 > 0.f, grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, near, s);
        return;
    }
    if (p2p_tpt() == 0) {
        const unsigned g2 = (grid + kP2PWarps - 1) / kP2PWarps;
        if (eps2 > 0.f)
            k_p2p_warp<true><<<g2, 32 * kP2PWarps, 0, s>>>(L, grid, leaves, sx, begin, end, offs, ids, far, perm, eps2, out);
        else
            k_p2p_warp<false><<<g2, 32 * kP2PWarps, 0, s>>>(L, grid, leaves, sx, begin, end, offs, ids, far, perm, eps2, out);
        note_launches(1);
        return;
    }
    switch (p2p_tpt()) {
    case 1: launch_p2p_t<1>(grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, s); break;
    case 2: launch_p2p_t<2>(grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, s); break;
    case 8: launch_p2p_t<8>(grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, s); break;
    case 4: launch_p2p_t<4>(grid, L, leaves, sx, begin, end, offs, ids, far, perm, eps2, out, s); break;
    }
}

void launch_p2p(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs,
                const int32_t *p2p_ids, const float4 *far, const uint32_t *perm, float eps2, float4 *out,
                cudaStream_t s)
{
    if (n <= 0) return;
    if (L >= 1 && p2p_tpt() == 20) {
        const unsigned grid = (unsigned)(int64_t(1) << (3 * (L - 1)));
        if (eps2 > 0.f)
            k_p2p_super<true><<<grid, kSuperThreads, 0, s>>>(L, sx, begin, end, far, perm, eps2, out);
        else
            k_p2p_super<false><<<grid, kSuperThreads, 0, s>>>(L, sx, begin, end, far, perm, eps2, out);
        note_launches(1);
        return;
    }
    dispatch_p2p((unsigned)(int64_t(1) << (3 * L)), L, nullptr, sx, begin, end, p2p_offs, p2p_ids, far, perm, eps2,
                 out, s);
}

void launch_p2p_cells(const int32_t *leaves, int64_t nleaves, int64_t n, const float4 *sx, const int32_t *begin,
                      const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, const float4 *far,
                      const uint32_t *perm, float eps2, float4 *out, cudaStream_t s)
{
    if (n <= 0 || nleaves <= 0) return;
    dispatch_p2p((unsigned)nleaves, 0, leaves, sx, begin, end, u_offs, u_ids, far, perm, eps2, out, s);
}

bool p2p_near_supported() { return p2p_has_near(); }

void launch_p2p_near(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end,
                     const uint32_t *p2p_offs, const int32_t *p2p_ids, float eps2, float4 *near, cudaStream_t s)
{
    if (n <= 0 || !p2p_has_near()) return;
    dispatch_p2p((unsigned)(int64_t(1) << (3 * L)), L, nullptr, sx, begin, end, p2p_offs, p2p_ids, nullptr, nullptr,
                 eps2, nullptr, s, near);
}

void launch_p2p_cells_near(const int32_t *leaves, int64_t nleaves, int64_t n, const float4 *sx, const int32_t *begin,
                           const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, float eps2, float4 *near,
                           cudaStream_t s)
{
    if (n <= 0 || nleaves <= 0 || !p2p_has_near()) return;
    dispatch_p2p((unsigned)nleaves, 0, leaves, sx, begin, end, u_offs, u_ids, nullptr, nullptr, eps2, nullptr, s, near);
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
