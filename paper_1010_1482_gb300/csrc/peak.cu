// Arithmetic-throughput probes used as roofline denominators: FP32 FFMA on the CUDA cores and
// the warp-level tensor-core MMA (TF32 m16n8k8, BF16 m16n8k16, FP32 accumulation).  Each
// kernel runs independent accumulation chains in registers only (one store per thread at the
// end), on a grid of 4 CTAs per SM, timed with CUDA events.
#include "common.cuh"
#include "gbfmm.h"

namespace gbfmm {

constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 4096;

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(float *out, float seed)
{
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = seed + i * threadIdx.x;
    const float m = 0.9999f, c = 1e-7f;
#pragma unroll 1
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] = fmaf(a[i], m, c);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_mma_tf32(float *out, float seed)
{
    uint32_t a[4], b[2];
    float d[8][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = __float_as_uint(seed + i);
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = __float_as_uint(seed - i);
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[c][i] = 0.f;
#pragma unroll 1
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
        for (int c = 0; c < 8; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_mma_bf16(float *out, float seed)
{
    uint32_t a[4], b[2];
    float d[8][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 0x3f803f80u + i;
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = 0x3f803f80u - i;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[c][i] = seed;
#pragma unroll 1
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
        for (int c = 0; c < 8; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace gbfmm

using namespace gbfmm;

extern "C" int gbfmm_probe_peak(int kind, double *tflops)
{
    if (!tflops || kind < 0 || kind > 2) return GBFMM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GBFMM_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 4 * sms;
    float *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kProbeThreads * sizeof(float)) != cudaSuccess) return GBFMM_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (kind == 0)
            k_probe_ffma<<<blocks, kProbeThreads>>>(out, 1.0f);
        else if (kind == 1)
            k_probe_mma_tf32<<<blocks, kProbeThreads>>>(out, 1.0f);
        else
            k_probe_mma_bf16<<<blocks, kProbeThreads>>>(out, 1.0f);
    };
    launch();  // warm-up
    cudaEventRecord(e0);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double threads = (double)blocks * kProbeThreads;
    double flop = 0.0;
    if (kind == 0)
        flop = threads * kProbeIters * 8 * 16 * 2.0;                     // FFMA = 2 flop
    else if (kind == 1)
        flop = threads / 32.0 * kProbeIters * 8 * (16.0 * 8 * 8 * 2);   // per warp-MMA
    else
        flop = threads / 32.0 * kProbeIters * 8 * (16.0 * 8 * 16 * 2);
    *tflops = flop * reps / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return cudaGetLastError() == cudaSuccess ? GBFMM_OK : GBFMM_ECUDA;
}
