// Measurement helpers exported next to the ABI: per-kernel CUDA-event timing of the
// evaluation launches, and pipe-throughput probes (MUFU sin/cos, FP32 FMA, FP64 FMA)
// used as the measured roofline denominators.  The paper has no counterpart; these
// exist so that the benchmark can time the dominant kernel on the stream it runs on.
#include <cuda_runtime.h>

#include <cstdint>

#include "rbe_context.h"

namespace rbe {

// Pipe probes: every thread runs `iters` rounds of 8 independent operations.
__global__ void k_probe_mufu(float* out, int iters, float seed)
{
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = seed + 0.01f * (threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float s;
            asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(v[j]));
            v[j] = s;
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j];
    if (acc == 12345.678f) out[0] = acc;
}

__global__ void k_probe_ffma(float* out, int iters, float seed)
{
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = seed + 0.01f * (threadIdx.x + j);
    const float a = 0.9999f, b = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaf(v[j], a, b);
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j];
    if (acc == 12345.678f) out[0] = acc;
}

__global__ void k_probe_dfma(float* out, int iters, float seed)
{
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = seed + 0.01 * (threadIdx.x + j);
    const double a = 0.9999, b = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fma(v[j], a, b);
    }
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j];
    if (acc == 12345.678) out[0] = (float)acc;
}

}  // namespace rbe

using namespace rbe;

extern "C" {

// Measures a pipe's throughput in operations per second (one sin.approx, FFMA or DFMA
// = one operation): kind 0 = MUFU sin, 1 = FP32 FMA, 2 = FP64 FMA.  Runs on the
// current device and the legacy default stream; synchronous.
rbe_status rbe_measure_pipe(int32_t kind, int32_t iters, double* ops_per_s)
{
    if (!ops_per_s || kind < 0 || kind > 2 || iters < 1) return RBE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RBE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RBE_ECUDA;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return RBE_ENOMEM;
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        if (kind == 0) k_probe_mufu<<<blocks, threads>>>(out, iters, 0.5f);
        else if (kind == 1) k_probe_ffma<<<blocks, threads>>>(out, iters, 0.5f);
        else k_probe_dfma<<<blocks, threads>>>(out, iters, 0.5f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return RBE_ECUDA;
    *ops_per_s = (double)blocks * threads * 8.0 * iters / (best * 1e-3);
    return RBE_OK;
}

}  // extern "C"
