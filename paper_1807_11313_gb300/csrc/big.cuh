// Global-memory 2-D FFT machinery and the all-pairs search body for N = 256
// (a per-CTA N x N work array in L2), shared by the kernels of k_big.cu and
// the multi-map kernel.
#pragma once
#include "common.cuh"

namespace bigk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kColTile = 8;

__device__ inline double block_sum_b(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < kWarps ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

__device__ inline float block_max_b(float v, float *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < kWarps ? sh[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    float r = sh[32];
    __syncthreads();
    return r;
}

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

// 2-D FFT of the N x N work array Z (global, row-major); sm holds
// max(kWarps * N, N * kColTile) complex values
template <int N>
__device__ void fft2_global(float2 *Z, float2 *sm, const float2 *tw) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2 *line = sm + w * N;
    for (int r = w; r < N; r += kWarps) {          // rows
        for (int i = lane; i < N; i += 32) line[i] = Z[(size_t)r * N + i];
        __syncwarp();
        warp_fft_line<N>(line, 1, tw);
        for (int i = lane; i < N; i += 32) Z[(size_t)r * N + i] = line[i];
        __syncwarp();
    }
    __syncthreads();
    for (int c0 = 0; c0 < N; c0 += kColTile) {     // columns, 8 at a time
        for (int i = threadIdx.x; i < N * kColTile; i += kThreads)
            sm[(i % kColTile) * N + i / kColTile] = Z[(size_t)(i / kColTile) * N + c0 + i % kColTile];
        __syncthreads();
        warp_fft_line<N>(sm + w * N, 1, tw);     // kWarps == kColTile: one column per warp
        __syncthreads();
        for (int i = threadIdx.x; i < N * kColTile; i += kThreads)
            Z[(size_t)(i / kColTile) * N + c0 + i % kColTile] = sm[(i % kColTile) * N + i / kColTile];
        __syncthreads();
    }
}

template <int N>
__device__ void make_tw(float2 *tw, int sign) {
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x)
        tw[k] = make_float2(kTwTable<N>.re[k], sign > 0 ? kTwTable<N>.im[k] : -kTwTable<N>.im[k]);
}

constexpr size_t smem_big(int N) { return sizeof(float2) * ((size_t)N * kColTile + N); }

// Z = X1 + i X2, X_j = conj(S_tj) S_p extended by Hermitian symmetry
template <int N>
__device__ void build_pair_big(float2 *Z, const float2 *__restrict__ t1, const float2 *__restrict__ t2,
                               const float2 *__restrict__ sp) {
    constexpr int HW = N / 2 + 1;
    for (int i = threadIdx.x; i < N * N; i += kThreads) {
        const int r = i / N, c = i % N;
        float2 z;
        if (c <= N / 2) {
            const int k = r * HW + c;
            const float2 s = sp[k];
            const float2 x1 = c_mulcj(t1[k], s), x2 = c_mulcj(t2[k], s);
            z = make_float2(x1.x - x2.y, x1.y + x2.x);
        } else {
            const int k = ((N - r) & (N - 1)) * HW + (N - c);
            const float2 s = sp[k];
            const float2 x1 = c_mulcj(t1[k], s), x2 = c_mulcj(t2[k], s);
            z = make_float2(x1.x + x2.y, -x1.y + x2.x);
        }
        Z[i] = z;
    }
}

// One work item: pattern p against slot pairs [pb, pe) on this CTA's N x N
// work array Z (global memory); sm / tw as in fft2_global (tw = inverse
// twiddles, already in place); folds the item's best into keys[p].
template <int N>
__device__ void search_body(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                            int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                            float2 *Z, float2 *sm, const float2 *tw, float *redf,
                            const int *__restrict__ cand, int kc) {
    constexpr int HW = N / 2 + 1;
    const int n = cand ? kc : T;
    const float2 *sp = Sp + (size_t)p * N * HW;
    float best_v = -INFINITY;
    int best_t = -1;
    for (int pi = pb; pi < pe; ++pi) {
        const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
        const int t1 = cand ? cand[(size_t)p * kc + j1] : j1;
        const int t2 = cand ? cand[(size_t)p * kc + j2] : j2;
        build_pair_big<N>(Z, St + (size_t)max(t1, 0) * N * HW, St + (size_t)max(t2, 0) * N * HW, sp);
        __syncthreads();
        fft2_global<N>(Z, sm, tw);
        float m1 = -INFINITY, m2 = -INFINITY;
        for (int i = threadIdx.x; i < N * N; i += kThreads) {
            const float2 z = Z[i];
            m1 = fmaxf(m1, z.x);
            m2 = fmaxf(m2, z.y);
        }
        m1 = block_max_b(m1, redf);
        m2 = block_max_b(m2, redf);
        if (t1 < 0) m1 = -INFINITY;
        if (t2 < 0) m2 = -INFINITY;
        if (t1 >= 0 && (m1 > best_v || (m1 == best_v && t1 < best_t))) { best_v = m1; best_t = t1; }
        if (j2 != j1 && t2 >= 0 && (m2 > best_v || (m2 == best_v && t2 < best_t))) { best_v = m2; best_t = t2; }
        if (peaks_all && threadIdx.x == 0) {
            peaks_all[(size_t)p * n + j1] = m1;
            if (j2 != j1) peaks_all[(size_t)p * n + j2] = m2;
        }
    }
    if (threadIdx.x == 0 && best_t >= 0) atomicMax(keys + p, pack_key(best_v, best_t));
}

}  // namespace bigk
