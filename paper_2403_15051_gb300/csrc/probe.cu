// Measured FP32 fused multiply-add throughput of the device: the denominator of the fused stage
// kernel's arithmetic roofline (the stage is bound by FP32 issue, not by HBM; the nominal rate,
// SMs x FP32 lanes x 2 x clock, is not what the chip sustains under load).
//
// Every thread runs kChains independent FMA chains (enough independent instructions in flight to
// cover the FMA latency on every scheduler); the grid fills every SM with two blocks of 1024
// threads.  The result of the chains is stored only if it takes an impossible value, so that the
// compiler keeps the arithmetic and no memory traffic enters the timed region.
#include <cuda_runtime.h>

#include "../../include/fdlb.h"

namespace fdlb {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ float g_probe_sink;

__global__ void __launch_bounds__(1024) ffma_probe_kernel(int iters, float seed) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * (float)(threadIdx.x + c);
    const float m = 0.9999f, k = 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.2345e30f) g_probe_sink = s;
}

}  // namespace
}  // namespace fdlb

// Runs the probe on the current device and stream: one warm-up launch, then `repeats` timed
// launches (CUDA events on `cuda_stream`); *tflops = the best rate (an FMA counted as two flops),
// *ms = that launch's duration.  FDLB_EINVAL for repeats < 1 or null outputs, FDLB_ECUDA /
// FDLB_ENOGPU from the runtime.
extern "C" int fdlb_fp32_fma_peak(void* cuda_stream, int repeats, double* tflops, double* ms) {
    using namespace fdlb;
    if (repeats < 1 || !tflops || !ms) return FDLB_EINVAL;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDLB_ENOGPU;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FDLB_ECUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int threads = 1024, blocks = 2 * n_sm, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FDLB_ECUDA;
    int rc = FDLB_OK;
    double best = 0.0, best_ms = 0.0;
    for (int r = 0; r <= repeats && rc == FDLB_OK; ++r) {
        cudaEventRecord(e0, s);
        ffma_probe_kernel<<<blocks, threads, 0, s>>>(iters, 1.0f + 1e-6f * (float)r);
        if (cudaPeekAtLastError() != cudaSuccess) rc = FDLB_ECUDA;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = FDLB_ECUDA;
        float t = 0.f;
        if (rc == FDLB_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = FDLB_ECUDA;
        if (rc == FDLB_OK && r > 0) {  // launch 0 warms up
            const double flops = 2.0 * kChains * kUnroll * (double)iters * threads * blocks;
            const double rate = flops / (t * 1e-3) / 1e12;
            if (rate > best) {
                best = rate;
                best_ms = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *tflops = best;
    *ms = best_ms;
    return FDLB_OK;
}
