// Normalised dot product (paper, Eq. 1 and the NDP section) and the
// peak-width measurement of the sampling-frequency section (Figs. 3, 4).
//
// k_ndp_norm: contrast normalisation of an N x N crop, one CTA per image.
//   The statistics are taken in one pass as sums of (x - x0) and (x - x0)^2
//   with x0 the crop's first pixel (a constant crop then gives exactly zero
//   variance, and the shift keeps the FP32 per-thread sums well conditioned),
//   combined across the block in FP64; the second pass re-reads the crop
//   (L1 / L2 resident) and writes v = (x - mean) / (sd N), so that a plain dot
//   product of two outputs is their NDP.  HBM: 4 B read and 4 + 2 B written
//   per pixel (FP32 and BF16 outputs).
// k_ndp_rescore: FP32 NDP of each pattern against its k candidates, the best
//   by (score desc, template asc).  HBM: 4 B per pixel of each candidate.
// k_fwhm: full width at half maximum of correlation-versus-angle curves, one
//   thread per curve.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kNormThreads = 256, kRescoreThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double *red) {
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // red may still be read by a previous call
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kNormThreads) k_ndp_norm(const float *__restrict__ img, long img_stride,
                                                           int row_stride, int ox, int oy, int n,
                                                           float *__restrict__ out32,
                                                           __nv_bfloat16 *__restrict__ out16,
                                                           int *__restrict__ degen) {
    __shared__ double red[kNormThreads / 32];
    const int p = blockIdx.x, tid = threadIdx.x;
    const long d = (long)n * n;
    const int lg = __ffs(n) - 1;   // n is a power of two
    const float *src = img + (size_t)p * img_stride + (size_t)oy * row_stride + ox;
    const float x0 = __ldg(src);
    float s1 = 0.f, s2 = 0.f;
    for (long i = tid; i < d; i += kNormThreads) {
        const float v = __ldg(src + (size_t)(i >> lg) * row_stride + (i & (n - 1))) - x0;
        s1 += v;
        s2 = fmaf(v, v, s2);
    }
    const double S1 = block_sum_d(s1, red), S2 = block_sum_d(s2, red);
    const double m1 = S1 / d, var = S2 / d - m1 * m1;
    const double mean = x0 + m1, sd = var > 0.0 ? sqrt(var) : 0.0;
    const bool bad = !(sd > 1e-12 * (1.0 + fabs(mean)));
    if (tid == 0 && degen) degen[p] = bad ? 1 : 0;
    const float m = (float)mean, scale = bad ? 0.f : (float)(1.0 / (sd * n));
    float *o32 = out32 ? out32 + (size_t)p * d : nullptr;
    __nv_bfloat16 *o16 = out16 ? out16 + (size_t)p * d : nullptr;
    for (long i = tid; i < d; i += kNormThreads) {
        const float v = bad ? 0.f : (__ldg(src + (size_t)(i >> lg) * row_stride + (i & (n - 1))) - m) * scale;
        if (o32) o32[i] = v;
        if (o16) o16[i] = __float2bfloat16_rn(v);
    }
}

__global__ void __launch_bounds__(kRescoreThreads) k_ndp_rescore(const float *__restrict__ pn,
                                                                 const float *__restrict__ tn, long d,
                                                                 const int *__restrict__ cand, int k,
                                                                 const int *__restrict__ degen,
                                                                 int *__restrict__ best,
                                                                 float *__restrict__ score) {
    __shared__ float red[kRescoreThreads / 32];
    const int p = blockIdx.x, tid = threadIdx.x;
    if (degen && degen[p]) {
        if (tid == 0) { best[p] = -1; score[p] = 0.f; }
        return;
    }
    const float4 *a = reinterpret_cast<const float4 *>(pn + (size_t)p * d);
    const long d4 = d / 4;
    int bt = -1;
    float bs = 0.f;
    for (int c = 0; c < k; ++c) {
        const int t = cand[(size_t)p * k + c];
        if (t < 0) continue;   // uniform across the block
        const float4 *b = reinterpret_cast<const float4 *>(tn + (size_t)t * d);
        float s = 0.f;
        for (long i = tid; i < d4; i += kRescoreThreads) {
            const float4 x = __ldg(a + i), y = __ldg(b + i);
            s = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, s))));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        float tot = 0.f;
#pragma unroll
        for (int w = 0; w < kRescoreThreads / 32; ++w) tot += red[w];
        if (bt < 0 || tot > bs || (tot == bs && t < bt)) { bt = t; bs = tot; }
    }
    if (tid == 0) { best[p] = bt; score[p] = bt < 0 ? 0.f : bs; }
}

// curves c < nc/2 read a, the others b; each [L] sampled at (j - (L-1)/2) step
__global__ void k_fwhm(const float *__restrict__ a, const float *__restrict__ b, int nc, int L, float step,
                       float *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const float *y = c < nc / 2 ? a + (size_t)c * L : b + (size_t)(c - nc / 2) * L;
    int m = 0;
    for (int j = 1; j < L; ++j)
        if (y[j] > y[m]) m = j;
    if (!(y[m] > 0.f)) { out[c] = -1.f; return; }
    const float h = 0.5f * y[m];
    int l = m, r = m;
    while (l > 0 && y[l - 1] >= h) --l;
    while (r < L - 1 && y[r + 1] >= h) ++r;
    if (l == 0 || r == L - 1) { out[c] = -1.f; return; }
    const float tl = (float)(l - 1) + (h - y[l - 1]) / (y[l] - y[l - 1]);
    const float tr = (float)r + (y[r] - h) / (y[r] - y[r + 1]);
    out[c] = (tr - tl) * step;
}

}  // namespace

cudaError_t launch_ndp_norm(const float *img, int P, long img_stride, int row_stride, int ox, int oy, int n,
                            float *out32, void *out16, int *degen, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (n < 16 || (n & (n - 1))) return cudaErrorInvalidValue;
    k_ndp_norm<<<P, kNormThreads, 0, st>>>(img, img_stride, row_stride, ox, oy, n, out32,
                                           static_cast<__nv_bfloat16 *>(out16), degen);
    return cudaGetLastError();
}

cudaError_t launch_ndp_rescore(const float *pn, const float *tn, long d, const int *cand, int k, const int *degen,
                               int P, int *best, float *score, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (d % 4 || k < 1) return cudaErrorInvalidValue;
    k_ndp_rescore<<<P, kRescoreThreads, 0, st>>>(pn, tn, d, cand, k, degen, best, score);
    return cudaGetLastError();
}

cudaError_t launch_fwhm(const float *a, const float *b, int nc, int L, float step, float *out, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    k_fwhm<<<(nc + 63) / 64, 64, 0, st>>>(a, b, nc, L, step, out);
    return cudaGetLastError();
}
