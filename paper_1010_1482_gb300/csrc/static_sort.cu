// gbfmm_sort_static: the Morton sort of the tree front end (root box, depth-L keys, stable
// radix sort, gather) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a host framework whose
// allocator owns every device byte, plug-ins that are handed only the buffers they read and
// write, or hooks that run while the application forbids allocation.  For them this entry
// point takes its scratch (ping-pong key / index buffers, the radix-sort histograms and look-back words,
// the root-box partials and completion counter) from one file-scope __device__ array of
// kStaticSortBytes.  Every GPU that loads the library holds that array until the process
// exits.  The caller still passes the input particles and the three outputs.
//
// The array's name is only a host-side stand-in in host code, so its device address is looked
// up with cudaGetSymbolAddress once per device (with that device current) on the first call
// there; that first call should therefore come before any stream capture.  The address is
// cached for the life of the process, so calls after cudaDeviceReset on that device are not
// supported.  All calls share the one array and it keeps the last call's contents: the
// completion counter and the status word are cleared at the start of every call, and calls
// that overlap on the GPU (two streams, or two host threads) race on the array.
//
// Only the uniform tree's keys (3L <= 30 bits, at most 4 radix passes of 8 bits) fit the
// array; the adaptive tree's 63-bit keys are refused before anything is launched.
#include "common.cuh"
#include "gbfmm.h"

#include <mutex>

namespace gbfmm {

constexpr int64_t kStaticSortMaxN = int64_t(1) << 20;

// scratch layout (byte offsets, each 256-aligned)
constexpr size_t kSsBox = 0;
constexpr size_t kSsCounter = 256;
constexpr size_t kSsStatus = 512;
constexpr size_t kSsPartials = 768;                                   // 304 x 8 floats
constexpr size_t kSsKeys = kSsPartials + 10240;                       // uint32[max n]
constexpr size_t kSsIdx = kSsKeys + 4 * kStaticSortMaxN;              // uint32[max n]
constexpr size_t kSsHist = kSsIdx + 4 * kStaticSortMaxN;              // radix-sort scratch (32-bit keys)
constexpr size_t kStaticSortBytes = kSsHist + sort_scratch_bytes(kStaticSortMaxN, 32);

static __device__ __align__(256) unsigned char g_sort_scratch[kStaticSortBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};
}  // namespace

}  // namespace gbfmm

using namespace gbfmm;

namespace {
bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}
}  // namespace

extern "C" int gbfmm_sort_static(const gbfmm_params *prm, int64_t n, const float *d_xyzq, float *d_sorted_xyzq,
                                 uint32_t *d_perm, uint32_t *d_sorted_leaf_keys, int32_t *d_status, void *stream)
{
    if (!prm || n < 0) return GBFMM_EINVAL;
    if (n > kStaticSortMaxN) return GBFMM_EUNSUPPORTED;
    int32_t L = 0;
    int rc = gbfmm_plan(prm, n, &L, nullptr);
    if (rc != GBFMM_OK) return rc;
    // the static array holds the 32-bit leaf keys of the uniform tree only
    if (prm->tree != GBFMM_TREE_UNIFORM) return GBFMM_EUNSUPPORTED;
    if (L < 0 || 3 * L > 30 || kSsHist + sort_scratch_bytes(n, 3 * L) > kStaticSortBytes) return GBFMM_EUNSUPPORTED;
    if (n == 0) return GBFMM_OK;
    if (!d_xyzq || !d_sorted_xyzq || !d_perm || !d_sorted_leaf_keys) return GBFMM_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_xyzq) % 16 || reinterpret_cast<uintptr_t>(d_sorted_xyzq) % 16)
        return GBFMM_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_perm) % 4 || reinterpret_cast<uintptr_t>(d_sorted_leaf_keys) % 4 ||
        reinterpret_cast<uintptr_t>(d_status) % 4)
        return GBFMM_EINVAL;
    {
        // every output is written while the input (and the other outputs, used as ping-pong
        // buffers) are read: no two of them may share a byte
        const size_t b16 = 16 * (size_t)n, b4 = 4 * (size_t)n;
        const void *ptr[5] = {d_xyzq, d_sorted_xyzq, d_perm, d_sorted_leaf_keys, d_status};
        const size_t len[5] = {b16, b16, b4, b4, d_status ? sizeof(int32_t) : 0};
        for (int i = 0; i < 5; ++i)
            for (int j = i + 1; j < 5; ++j)
                if (len[i] && len[j] && overlaps(ptr[i], len[i], ptr[j], len[j])) return GBFMM_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GBFMM_ECUDA;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return GBFMM_ECUDA;
            g_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Box *box = reinterpret_cast<Box *>(base + kSsBox);
    unsigned *counter = reinterpret_cast<unsigned *>(base + kSsCounter);
    // the status word the kernels raise: the caller's when given (so that it can be read
    // back), else the one in the static array
    int *status = d_status ? reinterpret_cast<int *>(d_status) : reinterpret_cast<int *>(base + kSsStatus);
    if (cudaMemsetAsync(base + kSsCounter, 0, 512, s) != cudaSuccess) return GBFMM_ECUDA;  // counter, status
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return GBFMM_ECUDA;
    const int passes = (3 * L + 7) / 8;
    // the sort ends in its first buffer pair after an even number of passes: start there with
    // the caller's outputs so the result lands in them
    uint32_t *k_caller = d_sorted_leaf_keys, *v_caller = d_perm;
    uint32_t *k_tmp = reinterpret_cast<uint32_t *>(base + kSsKeys), *v_tmp = reinterpret_cast<uint32_t *>(base + kSsIdx);
    uint32_t *k0 = (passes % 2 == 0) ? k_caller : k_tmp, *v0 = (passes % 2 == 0) ? v_caller : v_tmp;
    uint32_t *k1 = (passes % 2 == 0) ? k_tmp : k_caller, *v1 = (passes % 2 == 0) ? v_tmp : v_caller;
    const float4 *x = reinterpret_cast<const float4 *>(d_xyzq);
    launch_bbox(x, n, prm->has_box, prm->box_origin, prm->box_side, box,
                reinterpret_cast<float *>(base + kSsPartials), counter, status, s);
    launch_keys(x, n, box, L, k0, v0, s);
    uint32_t *kout = nullptr, *vout = nullptr;
    launch_sort_gather(k0, k1, v0, v1, n, 3 * L, base + kSsHist, status, x, reinterpret_cast<float4 *>(d_sorted_xyzq),
                       &kout, &vout, s);
    if (kout != k_caller || vout != v_caller) return GBFMM_ECUDA;  // buffer parity bookkeeping failed
    return cudaGetLastError() == cudaSuccess ? GBFMM_OK : GBFMM_ECUDA;
}
