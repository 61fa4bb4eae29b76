// Shared-memory line FFT (radix-2, one warp per line) and its twiddle table,
// used by the angular correlation of the refinement (k_eta_update).
#pragma once
#include "common.cuh"

namespace linefft {

// radix-2 FFT of one line of N points in shared memory (point i at x[i*es]),
// butterflies spread over the lanes of the calling warp
template <int N>
__device__ void warp_fft_line(float2 *x, int es, const float2 *tw) {
    constexpr int LOG = cx_log2(N);
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < N; i += 32) {
        const int j = __brev(i) >> (32 - LOG);
        if (i < j) {
            const float2 t = x[i * es];
            x[i * es] = x[j * es];
            x[j * es] = t;
        }
    }
    __syncwarp();
#pragma unroll 1
    for (int s = 0; s < LOG; ++s) {
        const int half = 1 << s;
        for (int b = lane; b < N / 2; b += 32) {
            const int k = b & (half - 1);
            const int i0 = ((b >> s) << (s + 1)) + k, i1 = i0 + half;
            const float2 w = tw[k << (LOG - 1 - s)];
            const float2 u = x[i0 * es], v = c_mul(x[i1 * es], w);
            x[i0 * es] = c_add(u, v);
            x[i1 * es] = c_sub(u, v);
        }
        __syncwarp();
    }
}

template <int N>
__device__ void make_tw(float2 *tw, int sign) {
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x)
        tw[k] = make_float2(kTwTable<N>.re[k], sign > 0 ? kTwTable<N>.im[k] : -kTwTable<N>.im[k]);
}

}  // namespace linefft
