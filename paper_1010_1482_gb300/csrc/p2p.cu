// P2P near field (Section "The P2P kernel implementation", Listings 1-2) and the direct
// all-pairs sum (Eq. 1), FP32 with the reciprocal square root.
//
// Pair rule (both kernels): with d = x_i - x_j and d2 = |d|^2,
//   phi_i  += q_j / sqrt(d2 + eps2),   grad_i -= q_j d / (d2 + eps2)^(3/2),
// and pairs with d2 == 0 (the particle itself, exact duplicates) contribute nothing.
//
// Decomposition (k_p2p_ws): one producer warp and four consumer warps per CTA; a CTA takes
// every gridDim.x-th target leaf.  The producer reads a leaf's neighbour rows (the uniform tree's
// <= 27 cells, or an adaptive leaf's U list), puts the leaf's own cell first, and copies the rows'
// particles with 1D bulk copies into one of two shared-memory stages while the consumers work on
// the other.  Each consumer thread holds two targets; when the leaf has fewer target slots than
// there are consumers the threads form G groups that split the sources round-robin, so the lanes
// stay busy for leaves of any occupancy (the paper instead pads targets to the block size).  Each
// thread sums its share in FP32; the group partials are combined per target with compensated
// (Kahan) summation.  Then either the far-field value is added the same way and the result
// written to the caller's original particle order, or (FMM) the compensated sums are stored for
// L2P, which adds the far field and writes the output.
#include "common.cuh"
#include "ptx.cuh"

#include <algorithm>

namespace gbfmm {

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

// Scalar pair rule of pair(), with the zero-distance test only where MASK (the target's own
// cell); the gradient accumulates +d q / r^3 and is negated once at the end.
template <bool SOFT, bool MASK>
GB_DEV void pairm(float xi, float yi, float zi, float4 s, float eps2, float &phi, float &gx, float &gy, float &gz)
{
    const float dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrt_ftz(SOFT ? d2 + eps2 : d2);
    if (MASK) inv = d2 > 0.f ? inv : 0.f;
    const float w = s.w * inv;
    phi += w;
    const float w3 = w * inv * inv;
    gx = fmaf(dx, w3, gx);
    gy = fmaf(dy, w3, gy);
    gz = fmaf(dz, w3, gz);
}

// ---- warp-specialised P2P: one producer warp stages, four consumer warps apply the pair rule ---
//
// A CTA takes the leaves blockIdx.x, blockIdx.x + gridDim.x, ...  The producer warp reads a
// leaf's neighbour rows (lane e holds row e of a block of up to 32: its first particle and count),
// moves the target's own cell to the front of its block (only its sources pay for the
// zero-distance test), scans the counts across the warp, and copies the rows' particles
// (contiguous float4 runs of the sorted array) with 1D bulk copies into one of two stage buffers
// of kP2PCap sources; the stage's full barrier completes when the bytes have landed.  The
// consumers apply the pair rule to a stage while the producer fills the other, so a leaf's list
// reads, row copies and the previous leaf's reduction overlap the pair loop.  Targets: 2 per
// consumer thread; when a leaf has fewer target slots than there are consumers the threads form G
// groups that take the staged sources round-robin; group partials are combined per target with
// compensated sums as before.  Every wait is bounded: on expiry the kernel raises kStatusTimeout,
// stops, and returns once its own copies have landed (bounded again).
constexpr int kP2PCap = 512;
constexpr int kP2PConsumers = 128;
constexpr int kP2PWsThreads = kP2PConsumers + 32;
constexpr int kP2PTargets = 2 * kP2PConsumers;  // targets per pass over the sources

struct P2PItem {
    int b0;     // the leaf's first particle (sorted order); -1 ends the stream
    int T;      // the leaf's particle count
    int tc;     // first target of this pass
    int chunk;  // sources staged (0: none, the pass only ends)
    int mend;   // leading staged sources of the target's own cell (zero-distance test)
    int flags;  // 1: first stage of the pass, 2: last stage of the pass, 4: targets are staged at tc
};

template <bool SOFT>
__global__ void __launch_bounds__(kP2PWsThreads, 8) k_p2p_ws(int L, const int32_t *__restrict__ leaves, Span lv,
                                                           int64_t nleaf, const float4 *__restrict__ sx,
                                                           const int32_t *__restrict__ begin,
                                                           const int32_t *__restrict__ end,
                                                           const uint32_t *__restrict__ p2p_offs,
                                                           const int32_t *__restrict__ p2p_ids,
                                                           const float4 *__restrict__ far,
                                                           const uint32_t *__restrict__ perm, float eps2,
                                                           float4 *__restrict__ out, float4 *__restrict__ near,
                                                           int *status)
{
    // two stages: the consumers read one while the producer's copies fill the other
    __shared__ __align__(128) float4 buf[2][kP2PCap];
    __shared__ float4 red[2][2][kP2PConsumers];
    __shared__ P2PItem item[2];
    __shared__ __align__(8) uint64_t full[2], empty[2], redbar[2];
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kP2PConsumers / 32);
            mbar_init(&redbar[k], kP2PConsumers);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int64_t count = leaves ? span_count(lv) : nleaf;

    if (tid >= kP2PConsumers) {  // ---------------- producer warp
        int stage = 0;
        uint32_t used = 0u, par = 0u;  // per stage: filled before; parity of its last fill
        bool ok = true;
        // claim the stage: wait until the consumers have released its previous fill
        auto claim = [&]() -> bool {
            if (((used >> stage) & 1u) &&
                !mbar_wait_bounded(&empty[stage], (par >> stage) & 1u, kWaitLimitNs, &abort_flag)) {
                abort_flag = 1;
                if (status) atomicOr(status, kStatusTimeout);
            }
            return !abort_flag;
        };
        auto advance = [&] {
            par = ((used >> stage) & 1u) ? par ^ (1u << stage) : par;
            used |= 1u << stage;
            stage ^= 1;
        };
        // publish one stage (lane 0); a stage with no sources completes on the arrival alone
        auto publish = [&](const P2PItem &v) {
            if (lane == 0) {
                item[stage] = v;
                if (v.chunk > 0)
                    mbar_expect_tx(&full[stage], (uint32_t)v.chunk * 16u);
                else
                    mbar_arrive(&full[stage]);
            }
            __syncwarp();
        };
        for (int64_t li = blockIdx.x; ok && li < count; li += gridDim.x) {
            const int64_t leaf = leaves ? (int64_t)leaves[li] : li;
            const int64_t g = leaves ? leaf : level_offset(L) + leaf;
            const int b0 = begin[g], T = end[g] - b0;
            if (T <= 0) continue;
            const uint32_t r0 = p2p_offs[leaf];
            const int nrow = (int)(p2p_offs[leaf + 1] - r0);
            for (int tc = 0; ok && tc < T; tc += kP2PTargets) {
                const int Tc = min(T - tc, kP2PTargets);
                bool emitted = false;
                for (int rb = 0; ok && rb < nrow; rb += 32) {
                    const int nr = min(32, nrow - rb);
                    const bool last_rb = rb + 32 >= nrow;
                    int cb = 0, cn = 0;
                    if (lane < nr) {
                        const int c = p2p_ids[r0 + rb + lane];
                        cb = begin[c];
                        cn = end[c] - cb;
                    }
                    // the target's own cell first
                    const unsigned self = __ballot_sync(~0u, lane < nr && cb == b0 && cn == T);
                    const int k = self ? __ffs(self) - 1 : 0;
                    const int cb0 = __shfl_sync(~0u, cb, 0), cn0 = __shfl_sync(~0u, cn, 0);
                    const int cbk = __shfl_sync(~0u, cb, k), cnk = __shfl_sync(~0u, cn, k);
                    if (self && k > 0) {
                        if (lane == 0) cb = cbk, cn = cnk;
                        else if (lane == k) cb = cb0, cn = cn0;
                    }
                    int incl = cn;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int v = __shfl_up_sync(~0u, incl, d);
                        if (lane >= d) incl += v;
                    }
                    const int pref = incl - cn, S = __shfl_sync(~0u, incl, 31);
                    const int nself = self ? T : 0;
                    for (int sc = 0; sc < S; sc += kP2PCap) {
                        const int chunk = min(kP2PCap, S - sc);
                        if (!claim()) {
                            ok = false;
                            break;
                        }
                        const bool last = last_rb && sc + kP2PCap >= S;
                        const bool staged = rb == 0 && sc == 0 && nself > 0 && tc + Tc <= chunk;
                        publish(P2PItem{b0, T, tc, chunk, max(0, min(chunk, nself - sc)),
                                        (emitted ? 0 : 1) | (last ? 2 : 0) | (staged ? 4 : 0)});
                        const int lo = max(pref, sc), hi = min(pref + cn, sc + chunk);
                        if (hi > lo)
                            tma_bulk_g2s(&buf[stage][lo - sc], &sx[cb + (lo - pref)], (uint32_t)(hi - lo) * 16u,
                                         &full[stage]);
                        emitted = true;
                        advance();
                    }
                    if (ok && last_rb && S == 0) {  // the pass ends on an empty block
                        if (!claim()) {
                            ok = false;
                            break;
                        }
                        publish(P2PItem{b0, T, tc, 0, 0, (emitted ? 0 : 1) | 2});
                        emitted = true;
                        advance();
                    }
                }
                if (ok && !emitted) {  // no neighbour rows at all
                    if (!claim()) {
                        ok = false;
                        break;
                    }
                    publish(P2PItem{b0, T, tc, 0, 0, 3});
                    advance();
                }
            }
        }
        if (ok && claim()) {  // end of stream
            publish(P2PItem{-1, 0, 0, 0, 0, 0});
            advance();
        }
        if (abort_flag) {
            // stopped early: return only once this warp's copies have landed
            for (int k = 0; k < 2; ++k)
                if ((used >> k) & 1u) mbar_wait_bounded(&full[k], ((par >> k) & 1u), kWaitLimitNs, nullptr);
        }
        return;
    }

    // -------------------------------------------------- consumer warps
    int stage = 0, rpar = 0;
    uint32_t fpar = 0u, rphase = 0u;  // per stage / per reduction buffer: parity of the next phase
    int slots = 1, G = 1, slot = 0, grp = 0, Tc = 0;
    float ax = 0.f, ay = 0.f, az = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    float pa = 0.f, gax = 0.f, gay = 0.f, gaz = 0.f, pb = 0.f, gbx = 0.f, gby = 0.f, gbz = 0.f;
    while (true) {
        if (!mbar_wait_bounded(&full[stage], (fpar >> stage) & 1u, kWaitLimitNs, &abort_flag) || abort_flag) {
            if (!abort_flag) {
                abort_flag = 1;
                if (status) atomicOr(status, kStatusTimeout);
            }
            return;
        }
        const P2PItem it = item[stage];
        if (it.b0 < 0) return;
        const float4 *src = buf[stage];
        if (it.flags & 1) {  // a new pass: its targets
            Tc = min(it.T - it.tc, kP2PTargets);
            slots = (Tc + 1) / 2;
            G = kP2PConsumers / slots;
            slot = tid % slots;
            grp = tid / slots;
            // a missing target repeats the slot's first one; its result is discarded
            const int ta = 2 * slot, tb = ta + 1 < Tc ? ta + 1 : ta;
            const float4 A = (it.flags & 4) ? src[it.tc + ta] : __ldg(&sx[it.b0 + it.tc + ta]);
            const float4 B = (it.flags & 4) ? src[it.tc + tb] : __ldg(&sx[it.b0 + it.tc + tb]);
            ax = A.x, ay = A.y, az = A.z, bx = B.x, by = B.y, bz = B.z;
            pa = gax = gay = gaz = pb = gbx = gby = gbz = 0.f;
        }
        if (grp < G) {
            int j = grp;
            for (; j < it.mend; j += G) {
                const float4 s4 = src[j];
                pairm<SOFT, true>(ax, ay, az, s4, eps2, pa, gax, gay, gaz);
                pairm<SOFT, true>(bx, by, bz, s4, eps2, pb, gbx, gby, gbz);
            }
#pragma unroll 4
            for (; j < it.chunk; j += G) {
                const float4 s4 = src[j];
                pairm<SOFT, false>(ax, ay, az, s4, eps2, pa, gax, gay, gaz);
                pairm<SOFT, false>(bx, by, bz, s4, eps2, pb, gbx, gby, gbz);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);
        fpar ^= 1u << stage;
        stage ^= 1;
        if (!(it.flags & 2)) continue;
        // end of the pass: combine the groups' partials per target.  red alternates between two
        // buffers, and every consumer waits for the pass's arrivals, so a pass's writes never
        // meet the previous pass's reads.
        red[rpar][0][tid] = make_float4(pa, -gax, -gay, -gaz);
        red[rpar][1][tid] = make_float4(pb, -gbx, -gby, -gbz);
        mbar_arrive(&redbar[rpar]);
        if (!mbar_wait_bounded(&redbar[rpar], (rphase >> rpar) & 1u, kWaitLimitNs, &abort_flag)) {
            if (!abort_flag) {
                abort_flag = 1;
                if (status) atomicOr(status, kStatusTimeout);
            }
            return;
        }
        rphase ^= 1u << rpar;
        if (grp == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = 2 * slot + h;
                if (t >= Tc) break;
                const int i = it.b0 + it.tc + t;
                Kahan a{0.f, 0.f}, kx{0.f, 0.f}, ky{0.f, 0.f}, kz{0.f, 0.f};
                for (int k = 0; k < G; ++k) {
                    const float4 v = red[rpar][h][k * slots + slot];
                    a.add(v.x);
                    kx.add(v.y);
                    ky.add(v.z);
                    kz.add(v.w);
                }
                if (near) {  // the compensated sums so far; the far field is added by L2P
                    near[2 * (int64_t)i] = make_float4(a.s, kx.s, ky.s, kz.s);
                    near[2 * (int64_t)i + 1] = make_float4(a.c, kx.c, ky.c, kz.c);
                    continue;
                }
                if (far) {
                    const float4 f = far[i];
                    a.add(f.x);
                    kx.add(f.y);
                    ky.add(f.z);
                    kz.add(f.w);
                }
                out[perm[i]] = make_float4(a.s, kx.s, ky.s, kz.s);
            }
        }
        rpar ^= 1;
    }
}

// ---- launchers --------------------------------------------------------------------------------
// CTAs resident per SM, and the largest shared-memory carveout so that the kernel's CTAs can
// share an SM with the far field's when both run at once
static int p2p_blocks_per_sm()
{
    static const int b = [] {
        cudaFuncSetAttribute(k_p2p_ws<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_p2p_ws<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_p2p_ws<false>, kP2PWsThreads, 0);
        return v > 0 ? v : 1;
    }();
    return b;
}

// nleaf: the leaves (uniform tree) or the capacity of the listed leaves (lv.cap).  Each CTA takes
// about kP2PLeavesPerCta of them (never fewer CTAs than fit on the GPU at once): enough leaves
// that the producer's staging of one hides behind the pair loop of another, few enough that CTAs
// retire often and the far field's kernels, beside P2P on the other stream, get SMs.  Measured on
// the 1M uniform step (p = 10): 1, 2, 4, 8 leaves and one persistent wave gave P2P 0.528, 0.520,
// 0.525, 0.541, 0.596 ms alone and 1.158, 1.152, 1.163, 1.189, 1.248 ms for the forked step; on
// 16M Plummer (p = 8) P2P took 8.91, 7.97, 9.29 ms with 1, 4 and one wave.
constexpr int kP2PLeavesPerCta = 4;
// the evaluating context's choice (gbfmm_set_p2p_leaves_per_cta, gbfmm_tune), set on entry to an
// evaluation by the thread that issues its launches; 0: kP2PLeavesPerCta
static thread_local int tl_leaves_per_cta = 0;
void set_p2p_leaves_per_cta(int leaves) { tl_leaves_per_cta = leaves; }

static void launch_leaf(int64_t nleaf, int L, const int32_t *leaves, const float4 *sx, const int32_t *begin,
                        const int32_t *end, const uint32_t *offs, const int32_t *ids, const float4 *far,
                        const uint32_t *perm, float eps2, float4 *out, float4 *near, int *status, cudaStream_t s,
                        Span lv = Span{})
{
    const int64_t resident = (int64_t)sm_count() * p2p_blocks_per_sm();
    const int lpc = tl_leaves_per_cta > 0 ? tl_leaves_per_cta : kP2PLeavesPerCta;
    int64_t grid = (nleaf + lpc - 1) / lpc;
    grid = std::min<int64_t>(nleaf, std::max<int64_t>(grid, resident));
    if (eps2 > 0.f)
        k_p2p_ws<true><<<(unsigned)grid, kP2PWsThreads, 0, s>>>(L, leaves, lv, nleaf, sx, begin, end, offs, ids, far,
                                                                 perm, eps2, out, near, status);
    else
        k_p2p_ws<false><<<(unsigned)grid, kP2PWsThreads, 0, s>>>(L, leaves, lv, nleaf, sx, begin, end, offs, ids, far,
                                                                  perm, eps2, out, near, status);
    note_launches(1);
}

void launch_p2p(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end, const uint32_t *p2p_offs,
                const int32_t *p2p_ids, const float4 *far, const uint32_t *perm, float eps2, float4 *out, int *status,
                cudaStream_t s)
{
    if (n <= 0) return;
    launch_leaf(int64_t(1) << (3 * L), L, nullptr, sx, begin, end, p2p_offs, p2p_ids, far, perm, eps2, out, nullptr,
                status, s);
}

void launch_p2p_cells(const int32_t *leaves, Span lv, int64_t n, const float4 *sx, const int32_t *begin,
                      const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, const float4 *far,
                      const uint32_t *perm, float eps2, float4 *out, int *status, cudaStream_t s)
{
    if (n <= 0 || lv.cap <= 0) return;
    launch_leaf(lv.cap, 0, leaves, sx, begin, end, u_offs, u_ids, far, perm, eps2, out, nullptr, status, s, lv);
}

bool p2p_near_supported() { return true; }

void launch_p2p_near(int L, int64_t n, const float4 *sx, const int32_t *begin, const int32_t *end,
                     const uint32_t *p2p_offs, const int32_t *p2p_ids, float eps2, float4 *near, int *status,
                     cudaStream_t s)
{
    if (n <= 0) return;
    launch_leaf(int64_t(1) << (3 * L), L, nullptr, sx, begin, end, p2p_offs, p2p_ids, nullptr, nullptr, eps2, nullptr,
                near, status, s);
}

void launch_p2p_cells_near(const int32_t *leaves, Span lv, int64_t n, const float4 *sx, const int32_t *begin,
                           const int32_t *end, const uint32_t *u_offs, const int32_t *u_ids, float eps2, float4 *near,
                           int *status, cudaStream_t s)
{
    if (n <= 0 || lv.cap <= 0) return;
    launch_leaf(lv.cap, 0, leaves, sx, begin, end, u_offs, u_ids, nullptr, nullptr, eps2, nullptr, near, status, s, lv);
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
