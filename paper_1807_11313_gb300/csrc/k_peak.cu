// FP32 FMA throughput of the device, measured: the denominator of the
// search kernels' roofline is 2 flops per FMA lane per clock (SMs x 128 lanes
// x 2 x clock), and this kernel shows what the FMA pipes actually sustain.
// Each thread runs eight independent FMA chains (enough to cover the FMA
// latency with the resident warps), so the kernel is bound by FMA issue alone.
#include "kernels.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024) k_fma_rate(int iters, float a, float b, float *sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) sink[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace

cudaError_t launch_fma_rate(int blocks, int threads, int iters, float *sink, cudaStream_t st) {
    k_fma_rate<<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-6f, sink);
    return cudaGetLastError();
}

double fma_rate_flops(int blocks, int threads, int iters) {
    return 2.0 * kChains * 16.0 * (double)iters * (double)blocks * (double)threads;
}
