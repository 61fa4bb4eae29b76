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
// k_bg_rows / k_bg_cols: background correction before the NDP, the crop minus
//   its separable Gaussian blur (rows through shared memory into a work array,
//   then 32-column strips of it).  HBM: about 20 B per pixel.
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

// ---- background correction: crop minus its separable Gaussian blur (weights
// exp(-k^2 / (2 sigma^2)), |k| <= R, normalised; edge pixels repeated)
constexpr int kBgRows = 8, kBgThreads = 256;

__device__ __forceinline__ void bg_weights(float *w, int R, float sigma) {
    const float c = -0.5f / (sigma * sigma);
    for (int k = threadIdx.x; k <= 2 * R; k += blockDim.x) w[k] = expf(c * (float)((k - R) * (k - R)));
    __syncthreads();
    // every thread sums the weights in the same order, so all hold the same total
    float s = 0.f;
    for (int k = 0; k <= 2 * R; ++k) s += w[k];
    __syncthreads();
    const float inv = 1.f / s;
    for (int k = threadIdx.x; k <= 2 * R; k += blockDim.x) w[k] *= inv;
    __syncthreads();
}

// rows: tmp [P][n][n] = horizontal blur of the crop; grid (n / kBgRows, P)
__global__ void __launch_bounds__(kBgThreads) k_bg_rows(const float *__restrict__ img, long img_stride,
                                                        int row_stride, int ox, int oy, int n, int R, float sigma,
                                                        float *__restrict__ tmp) {
    extern __shared__ float4 smem_raw[];
    float *w = reinterpret_cast<float *>(smem_raw);   // [2R + 1]
    float *rows = w + ((2 * R + 4) & ~3);              // [kBgRows][n]
    const int p = blockIdx.y, r0 = blockIdx.x * kBgRows, lg = __ffs(n) - 1;
    const float *src = img + (size_t)p * img_stride + (size_t)(oy + r0) * row_stride + ox;
    for (int i = threadIdx.x; i < kBgRows * n; i += kBgThreads)
        rows[i] = __ldg(src + (size_t)(i >> lg) * row_stride + (i & (n - 1)));
    bg_weights(w, R, sigma);
    float *dst = tmp + (size_t)p * n * n + (size_t)r0 * n;
    for (int i = threadIdx.x; i < kBgRows * n; i += kBgThreads) {
        const int r = i >> lg, c = i & (n - 1);
        const float *row = rows + r * n;
        float s = 0.f;
        if (c - R >= 0 && c + R < n) {
            for (int k = -R; k <= R; ++k) s = fmaf(w[k + R], row[c + k], s);
        } else {
            for (int k = -R; k <= R; ++k) s = fmaf(w[k + R], row[min(max(c + k, 0), n - 1)], s);
        }
        dst[i] = s;
    }
}

// columns: out [P][n][n] = crop - vertical blur of tmp; grid (n / 32, P),
// lane = column of a 32-wide strip, warp = row phase
__global__ void __launch_bounds__(kBgThreads) k_bg_cols(const float *__restrict__ img, long img_stride,
                                                        int row_stride, int ox, int oy, int n, int R, float sigma,
                                                        const float *__restrict__ tmp, float *__restrict__ out) {
    extern __shared__ float4 smem_raw[];
    float *w = reinterpret_cast<float *>(smem_raw);
    float *strip = w + ((2 * R + 4) & ~3);              // [n][32]
    const int p = blockIdx.y, c0 = blockIdx.x * 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *t = tmp + (size_t)p * n * n + c0;
    const int wdt = n < 32 ? n : 32;   // strip width (n = 16: half the lanes idle)
    for (int i = threadIdx.x; i < n * 32; i += kBgThreads)
        strip[i] = (i & 31) < wdt ? __ldg(t + (size_t)(i >> 5) * n + (i & 31)) : 0.f;
    bg_weights(w, R, sigma);
    if (lane >= wdt) return;
    const float *src = img + (size_t)p * img_stride + (size_t)oy * row_stride + ox + c0 + lane;
    float *dst = out + (size_t)p * n * n + c0 + lane;
    for (int r = warp; r < n; r += kBgThreads / 32) {
        float s = 0.f;
        if (r - R >= 0 && r + R < n) {
            for (int k = -R; k <= R; ++k) s = fmaf(w[k + R], strip[(r + k) * 32 + lane], s);
        } else {
            for (int k = -R; k <= R; ++k) s = fmaf(w[k + R], strip[min(max(r + k, 0), n - 1) * 32 + lane], s);
        }
        dst[(size_t)r * n] = __ldg(src + (size_t)r * row_stride) - s;
    }
}

// ---- the same blur with the truncation radius R fixed at compile time (the
// default sigma = N / 8 gives R = 3N / 8): the weights travel as a kernel
// parameter (constant bank, read as FMA operands of the unrolled taps) and
// every thread slides one window over J consecutive outputs, so a loaded
// pixel feeds up to J FMAs.
template <int R>
struct BgW {
    float w[2 * R + 1];
};

template <int N>
struct BgShape {
    static constexpr int J = N >= 64 ? 8 : N / 8;   // outputs per window
    static constexpr int LANES = N < 32 ? N : 32;   // rows (row pass) / columns (column pass) per CTA
    static constexpr int SPAN = N / 8;              // outputs of one warp along the blurred axis
};

// row pass: LANES rows per CTA, lane = row, the 8 warps split the columns;
// padded rows (edges repeated R times) in shared memory with an odd stride
template <int N, int R>
__global__ void __launch_bounds__(kBgThreads) k_bg_rows_t(const float *__restrict__ img, long img_stride,
                                                          int row_stride, int ox, int oy,
                                                          const __grid_constant__ BgW<R> W, float *__restrict__ tmp) {
    using S = BgShape<N>;
    constexpr int PW = N + 2 * R, LD = PW + 1, OLD = N + 1;
    extern __shared__ float4 smem_raw[];
    float *rows = reinterpret_cast<float *>(smem_raw);   // [LANES][LD]
    float *outs = rows + S::LANES * LD;                  // [LANES][OLD]
    const int p = blockIdx.y, r0 = blockIdx.x * S::LANES;
    const float *src = img + (size_t)p * img_stride + (size_t)(oy + r0) * row_stride + ox;
    for (int i = threadIdx.x; i < S::LANES * PW; i += kBgThreads) {
        const int r = i / PW, q = i % PW;
        rows[r * LD + q] = __ldg(src + (size_t)r * row_stride + min(max(q - R, 0), N - 1));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < S::LANES) {
        const float *row = rows + lane * LD;
        for (int c0 = warp * S::SPAN; c0 < (warp + 1) * S::SPAN; c0 += S::J) {
            float acc[S::J];
#pragma unroll
            for (int j = 0; j < S::J; ++j) acc[j] = 0.f;
#pragma unroll
            for (int m = 0; m < 2 * R + S::J; ++m) {
                const float v = row[c0 + m];
#pragma unroll
                for (int j = 0; j < S::J; ++j)
                    if (m - j >= 0 && m - j <= 2 * R) acc[j] = fmaf(W.w[m - j], v, acc[j]);
            }
#pragma unroll
            for (int j = 0; j < S::J; ++j) outs[lane * OLD + c0 + j] = acc[j];
        }
    }
    __syncthreads();
    float *dst = tmp + (size_t)p * N * N + (size_t)r0 * N;
    for (int i = threadIdx.x; i < S::LANES * N; i += kBgThreads) dst[i] = outs[(i / N) * OLD + i % N];
}

// column pass: a strip of LANES columns per CTA, lane = column, the 8 warps
// split the rows; padded strip (edge rows repeated R times) in shared memory
template <int N, int R>
__global__ void __launch_bounds__(kBgThreads) k_bg_cols_t(const float *__restrict__ img, long img_stride,
                                                          int row_stride, int ox, int oy,
                                                          const __grid_constant__ BgW<R> W,
                                                          const float *__restrict__ tmp, float *__restrict__ out) {
    using S = BgShape<N>;
    constexpr int PH = N + 2 * R, L = S::LANES;
    extern __shared__ float4 smem_raw[];
    float *strip = reinterpret_cast<float *>(smem_raw);   // [PH][L]
    const int p = blockIdx.y, c0 = blockIdx.x * L, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *t = tmp + (size_t)p * N * N + c0;
    for (int i = threadIdx.x; i < PH * L; i += kBgThreads) {
        const int q = i / L, c = i % L;
        strip[i] = __ldg(t + (size_t)min(max(q - R, 0), N - 1) * N + c);
    }
    __syncthreads();
    if (lane >= L) return;
    const float *src = img + (size_t)p * img_stride + (size_t)oy * row_stride + ox + c0 + lane;
    float *dst = out + (size_t)p * N * N + c0 + lane;
    for (int q0 = warp * S::SPAN; q0 < (warp + 1) * S::SPAN; q0 += S::J) {
        float acc[S::J];
#pragma unroll
        for (int j = 0; j < S::J; ++j) acc[j] = 0.f;
#pragma unroll
        for (int m = 0; m < 2 * R + S::J; ++m) {
            const float v = strip[(q0 + m) * L + lane];
#pragma unroll
            for (int j = 0; j < S::J; ++j)
                if (m - j >= 0 && m - j <= 2 * R) acc[j] = fmaf(W.w[m - j], v, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < S::J; ++j)
            dst[(size_t)(q0 + j) * N] = __ldg(src + (size_t)(q0 + j) * row_stride) - acc[j];
    }
}

template <int N, int R>
cudaError_t bg_fixed(const float *img, int P, long img_stride, int row_stride, int ox, int oy, float sigma,
                     float *tmp, float *out, cudaStream_t st) {
    using S = BgShape<N>;
    BgW<R> W;
    double w[2 * R + 1], sw = 0.0;
    for (int k = -R; k <= R; ++k) sw += (w[k + R] = exp(-(double)k * k / (2.0 * sigma * sigma)));
    for (int k = 0; k <= 2 * R; ++k) W.w[k] = (float)(w[k] / sw);
    const size_t sm_rows = sizeof(float) * S::LANES * ((N + 2 * R + 1) + (N + 1));
    const size_t sm_cols = sizeof(float) * (N + 2 * R) * S::LANES;
    cudaError_t e = cudaFuncSetAttribute(k_bg_rows_t<N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rows);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bg_cols_t<N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cols);
    if (e != cudaSuccess) return e;
    k_bg_rows_t<N, R><<<dim3(N / S::LANES, P), kBgThreads, sm_rows, st>>>(img, img_stride, row_stride, ox, oy, W, tmp);
    k_bg_cols_t<N, R><<<dim3(N / S::LANES, P), kBgThreads, sm_cols, st>>>(img, img_stride, row_stride, ox, oy, W, tmp,
                                                                          out);
    return cudaGetLastError();
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

cudaError_t launch_ndp_background(const float *img, int P, long img_stride, int row_stride, int ox, int oy, int n,
                                  float sigma, float *tmp, float *out, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (n < 16 || (n & (n - 1)) || !(sigma > 0.f) || sigma > (float)n) return cudaErrorInvalidValue;
    const int R = (int)(3.0f * sigma + 0.5f);
    // the radii of the default sigma = n / 8 run the compile-time kernels
    if (n == 16 && R == 6) return bg_fixed<16, 6>(img, P, img_stride, row_stride, ox, oy, sigma, tmp, out, st);
    if (n == 32 && R == 12) return bg_fixed<32, 12>(img, P, img_stride, row_stride, ox, oy, sigma, tmp, out, st);
    if (n == 64 && R == 24) return bg_fixed<64, 24>(img, P, img_stride, row_stride, ox, oy, sigma, tmp, out, st);
    if (n == 128 && R == 48) return bg_fixed<128, 48>(img, P, img_stride, row_stride, ox, oy, sigma, tmp, out, st);
    if (n == 256 && R == 96) return bg_fixed<256, 96>(img, P, img_stride, row_stride, ox, oy, sigma, tmp, out, st);
    const size_t wb = sizeof(float) * (size_t)((2 * R + 4) & ~3);
    const size_t sm_rows = wb + sizeof(float) * kBgRows * n, sm_cols = wb + sizeof(float) * 32 * n;
    cudaError_t e = cudaFuncSetAttribute(k_bg_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rows);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bg_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cols);
    if (e != cudaSuccess) return e;
    k_bg_rows<<<dim3(n / kBgRows, P), kBgThreads, sm_rows, st>>>(img, img_stride, row_stride, ox, oy, n, R, sigma,
                                                                   tmp);
    k_bg_cols<<<dim3((n + 31) / 32, P), kBgThreads, sm_cols, st>>>(img, img_stride, row_stride, ox, oy, n, R, sigma, tmp,
                                                              out);
    return cudaGetLastError();
}
