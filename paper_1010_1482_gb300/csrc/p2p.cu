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
// size).  Each thread sums its share in FP32; the group partials, and then the far-field
// value, are combined per target with compensated (Kahan) summation and written to the
// caller's original particle order.
#include "common.cuh"

namespace gbfmm {

constexpr int kP2PThreads = 128;
constexpr int kP2PTargetsPerThread = 2;
constexpr int kSrcCap = 1024;
constexpr int kRowCap = 32;

template <bool SOFT>
GB_DEV void pair(float xi, float yi, float zi, float4 s, float eps2, float &phi, float &gx, float &gy, float &gz)
{
    const float dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrtf(SOFT ? d2 + eps2 : d2);
    inv = d2 > 0.f ? inv : 0.f;
    const float qi = s.w * inv;
    phi += qi;
    const float qi3 = qi * inv * inv;
    gx = fmaf(-dx, qi3, gx);
    gy = fmaf(-dy, qi3, gy);
    gz = fmaf(-dz, qi3, gz);
}

struct Kahan {
    float s, c;
    GB_DEV void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

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

void launch_p2p(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs,
                const int32_t *p2p_ids, const float4 *far, const uint32_t *perm, float eps2, float4 *out,
                cudaStream_t s)
{
    if (n <= 0) return;
    unsigned grid = (unsigned)(int64_t(1) << (3 * L));
    constexpr int TPT = kP2PTargetsPerThread;
    if (eps2 > 0.f)
        k_p2p<true, TPT><<<grid, kP2PThreads, 0, s>>>(L, nullptr, sx, begin, end, p2p_offs, p2p_ids, far, perm, eps2,
                                                      out);
    else
        k_p2p<false, TPT><<<grid, kP2PThreads, 0, s>>>(L, nullptr, sx, begin, end, p2p_offs, p2p_ids, far, perm,
                                                       eps2, out);
    note_launches(1);
}

void launch_p2p_cells(const int32_t *leaves, int64_t nleaves, int64_t n, const float4 *sx, const int32_t *begin,
                      const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, const float4 *far,
                      const uint32_t *perm, float eps2, float4 *out, cudaStream_t s)
{
    if (n <= 0 || nleaves <= 0) return;
    constexpr int TPT = kP2PTargetsPerThread;
    if (eps2 > 0.f)
        k_p2p<true, TPT><<<(unsigned)nleaves, kP2PThreads, 0, s>>>(0, leaves, sx, begin, end, u_offs, u_ids, far, perm,
                                                                   eps2, out);
    else
        k_p2p<false, TPT><<<(unsigned)nleaves, kP2PThreads, 0, s>>>(0, leaves, sx, begin, end, u_offs, u_ids, far, perm,
                                                                    eps2, out);
    note_launches(1);
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
