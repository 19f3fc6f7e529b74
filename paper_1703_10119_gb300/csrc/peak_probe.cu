// Arithmetic-peak microbenchmarks (include/hygro_peaks.h): FP32 fused multiply-add (scalar and packed
// pairs), the MUFU approximate reciprocal and FP64 fused multiply-add, each as 8 independent dependency
// chains per thread over a grid of 4 blocks of 256 threads per SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hygro_peaks.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kBlock = 256;
constexpr int kBlocksPerSM = 4;

// Written only when a chain's result equals `never` (a value the chains cannot reach), which keeps the
// compiler from removing the chains.
__device__ double g_probe_sink;

__global__ void __launch_bounds__(kBlock) ffma_probe(int64_t iters, float a, float b, float never)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)threadIdx.x + (float)c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == never) g_probe_sink = s;
}

__global__ void __launch_bounds__(kBlock) ffma2_probe(int64_t iters, float a, float b, float never)
{
    uint64_t x[kChains], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float lo = 1e-3f * (float)threadIdx.x + (float)c, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == never) g_probe_sink = s;
}

// x <- rcp(x + b): the added term keeps two reciprocals in a row from cancelling (a reciprocal of a
// reciprocal could be folded away); the adds run on the FMA pipe, far from its limit at this rate.
__global__ void __launch_bounds__(kBlock) rcp_probe(int64_t iters, float a, float b, float never)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (float)threadIdx.x + (float)c + b * a;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                const float y = x[c] + b;
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(y));
            }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == never) g_probe_sink = s;
}

__global__ void __launch_bounds__(kBlock) dfma_probe(int64_t iters, double a, double b, double never)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (double)threadIdx.x + (double)c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == never) g_probe_sink = s;
}

cudaError_t launch(int32_t kind, int grid, cudaStream_t st, int64_t iters)
{
    // a < 1 and b small keep every chain bounded (x tends to b / (1 - a)); never = -1 is unreachable
    switch (kind) {
        case HYGRO_PEAK_FFMA: ffma_probe<<<grid, kBlock, 0, st>>>(iters, 0.9999f, 1e-4f, -1.0f); break;
        case HYGRO_PEAK_FFMA2: ffma2_probe<<<grid, kBlock, 0, st>>>(iters, 0.9999f, 1e-4f, -1.0f); break;
        case HYGRO_PEAK_RCP: rcp_probe<<<grid, kBlock, 0, st>>>(iters, 0.5f, 0.75f, -1.0f); break;
        default: dfma_probe<<<grid, kBlock, 0, st>>>(iters, 0.9999, 1e-4, -1.0); break;
    }
    return cudaGetLastError();
}

double ops_per_iter(int32_t kind) { return (double)kUnroll * kChains * (kind == HYGRO_PEAK_FFMA2 ? 2.0 : 1.0); }

}  // namespace

extern "C" HYGRO_API hygro_status hygro_peak_probe(int32_t kind, int32_t device, void *stream, double target_ms,
                                                   double *ops_per_s, double *ms)
{
    if (kind < HYGRO_PEAK_FFMA || kind > HYGRO_PEAK_DFMA || ops_per_s == nullptr || ms == nullptr ||
        !(target_ms >= 1.0 && target_ms <= 10000.0))
        return HYGRO_E_INVALID;
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return HYGRO_E_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return HYGRO_E_CUDA;
    const int grid = sms * kBlocksPerSM;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return HYGRO_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HYGRO_E_CUDA;
    }
    hygro_status rc = HYGRO_OK;
    float t = 0.0f;
    int64_t iters = 64;
    auto timed_launch = [&](int64_t n) -> bool {
        return cudaEventRecord(e0, st) == cudaSuccess && launch(kind, grid, st, n) == cudaSuccess &&
               cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
               cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
    };
    // warm-up; calibration launches, 8x longer each time, until one lasts 5 ms; the timed launch scaled
    // from the last calibration to target_ms
    if (!timed_launch(iters)) rc = HYGRO_E_CUDA;
    for (int pass = 0; pass < 8 && rc == HYGRO_OK; ++pass) {
        if (!timed_launch(iters)) {
            rc = HYGRO_E_CUDA;
            break;
        }
        if (t >= 5.0f) break;
        iters *= 8;
    }
    if (rc == HYGRO_OK) {
        const double scale = target_ms / (double)(t > 1e-3f ? t : 1e-3f);
        iters = (int64_t)((double)iters * (scale < 1.0 ? 1.0 : scale));
        if (!timed_launch(iters)) rc = HYGRO_E_CUDA;
    }
    if (rc == HYGRO_OK) {
        const double ops = ops_per_iter(kind) * (double)iters * (double)grid * kBlock;
        *ms = (double)t;
        *ops_per_s = ops / ((double)t * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
