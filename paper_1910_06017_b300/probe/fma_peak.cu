// fma_peak.cu -- the FP32 multiply-add throughput of the current GPU,
// measured, as the denominator of the LK kernel's roofline fraction.
//
// Every thread runs CHAINS independent multiply-add chains (enough to hide
// the pipeline latency), either scalar (fma.rn.f32) or packed two to an
// instruction (fma.rn.f32x2); the launch fills every SM with 8 CTAs of 256
// threads.  The time is taken with CUDA events on the launching stream
// after a warm-up launch; the result counts 2 flops per multiply-add.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;
constexpr int NT = 256;

__global__ void __launch_bounds__(NT) fma_scalar(int iters, float a, float b, float *sink) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 1.2345f) sink[blockIdx.x * NT + threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(NT) fma_packed(int iters, float a, float b, float *sink) {
    float2 x[CHAINS];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c].x + x[c].y;
    if (s == 1.2345f) sink[blockIdx.x * NT + threadIdx.x] = s;
}

}  // namespace

// FP32 TFLOP/s of `packed` ? fma_packed : fma_scalar over a launch of
// `iters` loop trips (8 CTAs of 256 threads per SM), and its duration in ms.
// Returns a negative value on a CUDA error.  `sink` is a device buffer of
// at least sms * 8 * 256 floats (never written in practice).
extern "C" double omt_probe_fma_tflops(int packed, int iters, float *sink, float *ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1.0;
    const int grid = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    const float a = 0.999999f, b = 1e-7f;
    auto launch = [&](int n) {
        if (packed) fma_packed<<<grid, NT>>>(n, a, b, sink);
        else fma_scalar<<<grid, NT>>>(n, a, b, sink);
    };
    launch(iters / 8 + 1);   // warm-up: clocks up, module loaded
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || ms <= 0.f) return -1.0;
    if (ms_out) *ms_out = ms;
    const double fmas = (double)grid * NT * (double)iters * UNROLL * CHAINS * (packed ? 2.0 : 1.0);
    return 2.0 * fmas / (ms * 1e-3) / 1e12;
}
