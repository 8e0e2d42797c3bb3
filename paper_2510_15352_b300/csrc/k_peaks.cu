// k_peaks.cu -- microbenchmarks of the SM arithmetic rates that bound the
// compositing kernel: FP32 fused multiply-add (scalar FFMA and the packed
// FP32x2 form) and the SFU base-2 exponential (ex2.approx.ftz.f32). The
// renderer's roofline divides its algorithmic flops by these measured rates
// instead of a figure derived from unit counts and the maximum clock.
//
// Every thread runs CHAINS independent dependency chains for `iters` rounds,
// enough to hide the pipe latency at full occupancy; the result is written
// only when it is impossible (x == 12345) so the work is not removed.
#include "gs.h"
#include "gs_internal.cuh"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 16;

__global__ void __launch_bounds__(PEAK_THREADS) k_peak_ffma(int iters, float seed, float *sink) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.001f * (threadIdx.x + c);
    const float m = 0.99993f, a = 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fmaf(x[c], m, a);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.0f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) k_peak_ffma2(int iters, float seed, float *sink) {
    float2 x[CHAINS / 2];
#pragma unroll
    for (int c = 0; c < CHAINS / 2; ++c)
        x[c] = make_float2(seed + 0.001f * (threadIdx.x + c), seed - 0.001f * c);
    const float2 m = make_float2(0.99993f, 0.99991f), a = make_float2(1e-4f, 2e-4f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < CHAINS / 2; ++c) x[c] = __ffma2_rn(x[c], m, a);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS / 2; ++c) s += x[c].x + x[c].y;
    if (s == 12345.0f) sink[blockIdx.x] = s;
}

__device__ __forceinline__ float ex2_neg(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

__global__ void __launch_bounds__(PEAK_THREADS) k_peak_ex2(int iters, float seed, float *sink) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.01f * c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = ex2_neg(x[c]);  // stays in (0, 1]
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.0f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" gs_status gs_microbench(int32_t kind, int32_t blocks, int32_t iters, float *sink,
                                   int64_t *ops, void *stream) {
    if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !sink || !ops)
        return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long per_thread = (long long)iters * 8 * CHAINS;  // FMAs or ex2 per thread
    const long long threads = (long long)blocks * PEAK_THREADS;
    switch (kind) {
        case 0: k_peak_ffma<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.5f, sink); break;
        case 1: k_peak_ffma2<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.5f, sink); break;
        default: k_peak_ex2<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.5f, sink); break;
    }
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    // flops (2 per FMA) for the FMA kernels, exponentials for ex2
    *ops = kind == 2 ? per_thread * threads : 2 * per_thread * threads;
    return GS_OK;
}
