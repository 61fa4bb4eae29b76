// Up-sampled correlation peak: the paper refines the integer peak by
// "up-sampling" (its method is in an absent reference); here the correlation
// is evaluated off the integer grid by its Fourier series, as in
// matrix-multiply DFT up-sampling.
//
// For pattern p with template t and cross-power half spectrum
// X[u][v] = conj(S_t[u][v]) S_p[u][v] (v = 0..N/2), the real surface off the
// grid is r(y, x) = sum_v w_v Re(sum_u X[u][v] e^{+2 pi i (f(u) y + v x) / N}),
// w_0 = w_{N/2} = 1, w_v = 2 otherwise, f(u) the signed frequency; at integer
// shifts this is the FFT surface.  It is evaluated on the (2U+1)^2 grid
// y0 + (m - U)/U, x0 + (l - U)/U around the integer argmax (y0, x0) as two
// small matrix products: T1[m][v] = sum_u E[m][u] X[u][v] (each thread one
// column v, the column read coalesced across threads), then
// r[m][l] = sum_v w_v Re(T1[m][v] F[l][v]); the grid argmax (ties: lowest
// (m, l) row-major) replaces the peak and the shift.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kUpThreads = 256, kMaxU = 20, kMaxM = 2 * kMaxU + 1;

// e^{+2 pi i (k0 / N + num / den)} with k0 an integer and num / den a small rational
__device__ __forceinline__ float2 phase(int k0, int N, int num, int den) {
    const float a = 2.f * (float)(((k0 % N) + N) % N) / N + 2.f * (float)num / (float)den;   // in units of pi
    float s, c;
    sincospif(a, &s, &c);
    return make_float2(c, s);
}

template <int N>
__global__ void __launch_bounds__(kUpThreads) k_upsample_peak(const float2 *__restrict__ St,
                                                              const int *__restrict__ tidx,
                                                              const float2 *__restrict__ Sp,
                                                              const int *__restrict__ degen,
                                                              const int *__restrict__ active, int U,
                                                              const int *__restrict__ argmax,
                                                              float *__restrict__ peak, float *__restrict__ shift) {
    constexpr int HW = N / 2 + 1;
    const int p = blockIdx.x, tid = threadIdx.x, M = 2 * U + 1;
    if (active && !active[p]) return;
    const int t = tidx ? tidx[p] : p;
    if ((degen && degen[p]) || t < 0) return;   // the integer peak kernel wrote zeros
    extern __shared__ float4 smem_raw[];
    float2 *E = reinterpret_cast<float2 *>(smem_raw);   // [M][N]  e^{2 pi i f(u) y_m / N}
    float2 *F = E + (size_t)M * N;                      // [M][HW] e^{2 pi i v x_l / N}
    float2 *T1 = F + (size_t)M * HW;                    // [M][HW]
    __shared__ float bv_w[kUpThreads / 32];
    __shared__ int bi_w[kUpThreads / 32];
    const int i0 = argmax[p], y0 = i0 / N, x0 = i0 % N;
    for (int i = tid; i < M * N; i += kUpThreads) {
        const int m = i / N, u = i % N, fu = u < N / 2 ? u : u - N;
        E[i] = phase(fu * y0, N, fu * (m - U), U * N);
    }
    for (int i = tid; i < M * HW; i += kUpThreads) {
        const int l = i / HW, v = i % HW;
        F[i] = phase(v * x0, N, v * (l - U), U * N);
    }
    __syncthreads();
    // T1[m][v] = sum_u E[m][u] X[u][v]: thread v holds the M accumulators of its column
    const float2 *st = St + (size_t)t * N * HW, *sp = Sp + (size_t)p * N * HW;
    for (int v = tid; v < HW; v += kUpThreads) {
        float2 acc[kMaxM];
#pragma unroll
        for (int m = 0; m < kMaxM; ++m) acc[m] = make_float2(0.f, 0.f);
        for (int u = 0; u < N; ++u) {
            const float2 x = c_mulcj(__ldg(st + (size_t)u * HW + v), __ldg(sp + (size_t)u * HW + v));
#pragma unroll
            for (int m = 0; m < kMaxM; ++m)
                if (m < M) {
                    const float2 e = E[m * N + u];
                    acc[m].x = fmaf(e.x, x.x, fmaf(-e.y, x.y, acc[m].x));
                    acc[m].y = fmaf(e.x, x.y, fmaf(e.y, x.x, acc[m].y));
                }
        }
#pragma unroll
        for (int m = 0; m < kMaxM; ++m)
            if (m < M) T1[m * HW + v] = acc[m];
    }
    __syncthreads();
    // r[m][l] and its argmax
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int i = tid; i < M * M; i += kUpThreads) {
        const int m = i / M, l = i % M;
        float s = 0.f;
        for (int v = 0; v < HW; ++v) {
            const float2 a = T1[m * HW + v], f = F[l * HW + v];
            const float re = a.x * f.x - a.y * f.y;
            s = fmaf((v == 0 || v == N / 2) ? 1.f : 2.f, re, s);
        }
        if (s > bv || (s == bv && i < bi)) { bv = s; bi = i; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { bv_w[tid >> 5] = bv; bi_w[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kUpThreads / 32; ++w)
            if (bv_w[w] > bv || (bv_w[w] == bv && bi_w[w] < bi)) { bv = bv_w[w]; bi = bi_w[w]; }
        const int m = bi / M, l = bi % M;
        peak[p] = bv;
        shift[2 * p] = (float)(x0 < N / 2 ? x0 : x0 - N) + (float)(l - U) / U;
        shift[2 * p + 1] = (float)(y0 < N / 2 ? y0 : y0 - N) + (float)(m - U) / U;
    }
}

template <int N>
cudaError_t upsample_n(const float2 *St, const int *tidx, const float2 *Sp, const int *degen, const int *active,
                       int P, int U, const int *argmax, float *peak, float *shift, cudaStream_t st) {
    const int M = 2 * U + 1, HW = N / 2 + 1;
    const size_t sm = sizeof(float2) * ((size_t)M * N + 2 * (size_t)M * HW);
    cudaError_t e = cudaFuncSetAttribute(k_upsample_peak<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_upsample_peak<N><<<P, kUpThreads, sm, st>>>(St, tidx, Sp, degen, active, U, argmax, peak, shift);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_upsample_peak(int N, const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                 const int *active, int P, int U, const int *argmax, float *peak, float *shift,
                                 cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (U < 2 || U > kMaxU) return cudaErrorInvalidValue;
    switch (N) {
        case 16: return upsample_n<16>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 32: return upsample_n<32>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 64: return upsample_n<64>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 128: return upsample_n<128>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 96: return upsample_n<96>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 160: return upsample_n<160>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 200: return upsample_n<200>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        case 256: return upsample_n<256>(St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
        default: return cudaErrorInvalidValue;
    }
}
