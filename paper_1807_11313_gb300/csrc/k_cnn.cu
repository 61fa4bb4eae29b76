// Learned orientation proposal: forward and backward kernels of the small
// convolutional network, its Gram-Schmidt heads with the cubic-symmetric
// winner-takes-all loss, Adam, and the proposal bookkeeping.
//
// The paper indexes by template matching alone; the network is an extension
// that proposes k orientations per pattern, each then scored by the paper's
// cross-correlation (Fig. 1 B-C) and refined (Fig. 6).  Architecture: per
// pattern standardisation (as in the pre-processing before correlation),
// five 3 x 3 stride-2 convolutions with bias and ReLU (1 -> 32 -> 64 -> 64 ->
// 128 -> 128 channels, 128 -> 4 px), mean pool, fc 128 -> 256 + ReLU, fc
// 256 -> 6k; head h turns (a1, a2) into R = [b1 b2 b3] by Gram-Schmidt (the
// continuous 6-D representation of Zhou et al. 2019).
//
// Every layer is a tiled FP32 matrix product whose operand loaders gather
// from the activations directly (implicit im2col), so no unfolded copy is
// written: C[m][n] = sum_k A(m, k) B(k, n) with the layer's loaders and
// epilogue.  Weight gradients split the long reduction over gridDim.z and
// accumulate with atomics.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

template <class LA, class LB, class EP>
__global__ void __launch_bounds__(GT) k_gemm(int M, int N, int K, int kper, LA la, LB lb, EP ep) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kper, ke = min(K, kb + kper);
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + i * GT;
            const int am = e / BK, ak = e % BK;       // A: consecutive threads walk k
            const int m = m0 + am, k = k0 + ak;
            As[ak][am] = (m < M && k < ke) ? la(m, k) : 0.f;
            const int bk = e / BN, bn = e % BN;       // B: consecutive threads walk n
            const int n = n0 + bn, kk = k0 + bk;
            Bs[bk][bn] = (n < N && kk < ke) ? lb(kk, n) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) ep(m, n, acc[i][j]);
        }
}

// the reduction length per split (a multiple of BK) for about `splits` splits of K
int split_kper(int K, int splits) {
    const int kchunks = (K + BK - 1) / BK;
    splits = max(1, min(splits, kchunks));
    return ((kchunks + splits - 1) / splits) * BK;
}

template <class LA, class LB, class EP>
cudaError_t gemm_kper(int M, int N, int K, int kper, LA la, LB lb, EP ep, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const int splits = (K + kper - 1) / kper;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    k_gemm<<<grid, GT, 0, st>>>(M, N, K, kper, la, lb, ep);
    return cudaGetLastError();
}
template <class LA, class LB, class EP>
cudaError_t gemm(int M, int N, int K, int splits, LA la, LB lb, EP ep, cudaStream_t st) {
    return gemm_kper(M, N, K, split_kper(K, splits), la, lb, ep, st);
}

// reduction splits so that a weight-gradient launch has about two CTAs per SM
int grad_splits(int M, int N, int K, int num_sms) {
    const long tiles = (long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const long want = (2L * num_sms + tiles - 1) / tiles;
    return (int)max(1L, min(want, (long)(K + 4 * BK - 1) / (4 * BK)));
}

// ------------------------------------------------------------- loaders
struct Src {   // layer input: activations [B][C][S][S], or the raw patterns (layer 1)
    const float *x;
    int C, S;
    long img_stride, row_stride;   // floats between images / rows
    int ox, oy;                    // crop offsets (layer 1)
    const float2 *affine;          // per-image (scale, shift) of the standardisation, or null
};

// im2col element (k = ci*9 + ky*3 + kx, n = b*So*So + oy*So + ox)
__device__ __forceinline__ float im2col(const Src &s, int So, int k, int n) {
    const int ci = k / 9, r = k - ci * 9, ky = r / 3, kx = r - ky * 3;
    const int lg = __ffs(So) - 1;   // output sides are powers of two: shifts, not divisions
    const int b = n >> (2 * lg), p = n & (So * So - 1), oy = p >> lg, ox = p & (So - 1);
    const int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
    if (iy < 0 || iy >= s.S || ix < 0 || ix >= s.S) return 0.f;
    const float v = s.x[b * s.img_stride + (long)ci * s.S * s.S + (long)(s.oy + iy) * s.row_stride + s.ox + ix];
    if (!s.affine) return v;
    const float2 a = s.affine[b];
    return fmaf(v, a.x, a.y);
}

struct LoadW {   // weights [M][K] row-major (conv W[co][ci*9] or fc W[out][in])
    const float *w;
    int K;
    __device__ float operator()(int m, int k) const { return w[(long)m * K + k]; }
};
struct LoadWT {   // transposed weights: A(m, k) = W[k][m] of a [K][M] matrix
    const float *w;
    int M;
    __device__ float operator()(int m, int k) const { return w[(long)k * M + m]; }
};
struct LoadWconvT {   // A(m = ci, k = co*9 + r) = W[co][ci][r] of conv weights [Co][Ci][9]
    const float *w;
    int Ci;
    __device__ float operator()(int m, int k) const {
        const int co = k / 9, r = k - co * 9;
        return w[((long)co * Ci + m) * 9 + r];
    }
};
struct LoadIm2col {
    Src s;
    int So;
    __device__ float operator()(int k, int n) const { return im2col(s, So, k, n); }
};
struct LoadIm2colT {   // B(k = (b, p), n = ci*9 + ...) for the weight gradient
    Src s;
    int So;
    __device__ float operator()(int k, int n) const { return im2col(s, So, n, k); }
};
struct LoadGradT {   // A(m = co, k = (b, p)) = g[b][co][p]
    const float *g;
    int C, Q;
    __device__ float operator()(int m, int k) const {
        const int b = k >> (__ffs(Q) - 1), p = k & (Q - 1);   // Q is a power of two
        return g[((long)b * C + m) * Q + p];
    }
};
// dX gather: B(k = co*9 + ky*3 + kx, n = b*Si*Si + iy*Si + ix) = g[b][co][oy][ox]
// where iy = 2 oy - 1 + ky (zero where no such output exists)
struct LoadGradScatter {
    const float *g;
    int Co, So;
    __device__ float operator()(int k, int n) const {
        const int Si = 2 * So;
        const int co = k / 9, r = k - co * 9, ky = r / 3, kx = r - ky * 3;
        const int lg = __ffs(Si) - 1;   // a power of two
        const int b = n >> (2 * lg), p = n & (Si * Si - 1), iy = p >> lg, ix = p & (Si - 1);
        const int ty = iy + 1 - ky, tx = ix + 1 - kx;
        if (ty < 0 || tx < 0 || (ty & 1) || (tx & 1)) return 0.f;
        const int oy = ty >> 1, ox = tx >> 1;
        if (oy >= So || ox >= So) return 0.f;
        return g[(((long)b * Co + co) * So + oy) * So + ox];
    }
};
struct LoadRows {   // B(k, n) = X[n][k] of a row-major [N][K] matrix (a batch of vectors)
    const float *x;
    int K;
    __device__ float operator()(int k, int n) const { return x[(long)n * K + k]; }
};
struct LoadRowsT {   // A(m, k) = X[k][m] of a row-major [K][M] matrix
    const float *x;
    int M;
    __device__ float operator()(int m, int k) const { return x[(long)k * M + m]; }
};
struct LoadRowsB {   // B(k, n) = X[k][n] of a row-major [K][N] matrix
    const float *x;
    int N;
    __device__ float operator()(int k, int n) const { return x[(long)k * N + n]; }
};

// ----------------------------------------------------------- epilogues
struct EpConv {   // y[b][co][p] = relu(acc + bias[co])
    float *y;
    const float *bias;
    int Co, Q;
    __device__ void operator()(int m, int n, float v) const {
        const int b = n >> (__ffs(Q) - 1), p = n & (Q - 1);   // Q is a power of two
        y[((long)b * Co + m) * Q + p] = fmaxf(v + bias[m], 0.f);
    }
};
struct EpVec {   // y[n][m] = act(acc + bias[m]) for a batch of vectors
    float *y;
    const float *bias;
    int M;
    bool relu;
    __device__ void operator()(int m, int n, float v) const {
        v += bias[m];
        y[(long)n * M + m] = relu ? fmaxf(v, 0.f) : v;
    }
};
struct EpMasked {   // y[n][m] = acc * (mask[n][m] > 0) (gradient through a ReLU)
    float *y;
    const float *mask;
    int M;
    __device__ void operator()(int m, int n, float v) const {
        const long i = (long)n * M + m;
        y[i] = mask[i] > 0.f ? v : 0.f;
    }
};
struct EpMaskedImg {   // gx[b][ci][p] = acc * (a[b][ci][p] > 0), n = b*Q + p
    float *y;
    const float *mask;
    int C, Q;
    __device__ void operator()(int m, int n, float v) const {
        const int b = n >> (__ffs(Q) - 1), p = n & (Q - 1);   // Q is a power of two
        const long i = ((long)b * C + m) * Q + p;
        y[i] = mask[i] > 0.f ? v : 0.f;
    }
};
struct EpStore {   // y[n][m] = acc
    float *y;
    int M;
    __device__ void operator()(int m, int n, float v) const { y[(long)n * M + m] = v; }
};
struct EpPartial {   // part[split][m][n] = acc (split = blockIdx.z; summed in split order afterwards)
    float *part;
    int M, N;
    __device__ void operator()(int m, int n, float v) const {
        part[((long)blockIdx.z * M + m) * N + n] = v;
    }
};

// out[i] = sum over z of part[z][i], z in increasing order (fixed order: the
// same inputs give the same sums on every run)
__global__ void k_sum_partials(const float *__restrict__ part, int splits, long n, float *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float s = part[i];
        for (int z = 1; z < splits; ++z) s += part[(long)z * n + i];
        out[i] = s;
    }
}

// ------------------------------------------------------ small kernels
// per-pattern (scale, shift) of the standardisation of the crop: (x - mean) / std
__global__ void k_cnn_stats(const float *__restrict__ x, long img_stride, long row_stride, int ox, int oy,
                            int S, float2 *__restrict__ affine) {
    // FP32 partial sums of (v - v0), v0 the first pixel (a constant image has exactly zero
    // variance; the shift keeps the partial sums well conditioned), combined in FP64
    const float *img = x + blockIdx.x * img_stride + (long)oy * row_stride + ox;
    const int lg = __ffs(S) - 1;   // S is a power of two
    const float v0 = img[0];
    float s = 0.f, s2 = 0.f;
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
        const float d = img[(long)(i >> lg) * row_stride + (i & (S - 1))] - v0;
        s += d;
        s2 = fmaf(d, d, s2);
    }
    __shared__ double r1[32], r2[32];
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += r1[w];
            b += r2[w];
        }
        const double n = (double)S * S, m1 = a / n, mean = v0 + m1;
        const double var = fmax(b / n - m1 * m1, 0.0), sd = sqrt(var);
        const bool degenerate = !(sd > 1e-12 * (1.0 + fabs(mean)));
        affine[blockIdx.x] = degenerate ? make_float2(0.f, 0.f) : make_float2((float)(1.0 / sd), (float)(-mean / sd));
    }
}

// mean over the Q positions of each channel: pool[b][c]
__global__ void k_cnn_pool(const float *__restrict__ a, int BC, int Q, float *__restrict__ pool) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BC) return;
    float s = 0.f;
    for (int p = 0; p < Q; ++p) s += a[(long)i * Q + p];
    pool[i] = s / Q;
}

// ---- BF16 inference form: the first convolution (K = 9) stays an FP32
// product and writes BF16 NHWC activations; convolutions 2..5 run as implicit
// GEMMs on the tensor cores (k_conv.cu) on BF16 NHWC activations and BF16
// weights [Co][Kp] (K = 9 Ci in the order (ky * 3 + kx) Ci + ci, padded with
// zeros to Kp, a multiple of 64), bias and ReLU in their epilogue.

// the first convolution (one input channel, 32 outputs) directly: one thread
// per output position, the standardised 3 x 3 input window against all 32
// filters (weights and biases in shared memory), bias, ReLU, NHWC output
// rounded to BF16 (the second convolution's operand)
__global__ void __launch_bounds__(256) k_cnn_conv1_nhwc(const float *__restrict__ x, long img_stride,
                                                        long row_stride, int ox0, int oy0,
                                                        const float2 *__restrict__ affine,
                                                        const float *__restrict__ w, const float *__restrict__ bias,
                                                        int B, __nv_bfloat16 *__restrict__ y) {
    constexpr int S = 128, So = 64, Co = 32;
    __shared__ __align__(16) float ws[9 * Co];   // [tap][channel]: four channels per 16-byte broadcast load
    __shared__ float bs[Co];
    for (int i = threadIdx.x; i < Co * 9; i += blockDim.x) ws[(i % 9) * Co + i / 9] = w[i];
    if (threadIdx.x < Co) bs[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long)B * So * So) return;
    const int b = (int)(n >> 12), p = (int)(n & 4095), oy = p >> 6, ox = p & 63;
    const float2 a = affine[b];
    const float *img = x + b * img_stride + (long)oy0 * row_stride + ox0;
    float v[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int iy = 2 * oy - 1 + r / 3, ix = 2 * ox - 1 + r % 3;
        v[r] = (iy >= 0 && iy < S && ix >= 0 && ix < S) ? fmaf(img[(long)iy * row_stride + ix], a.x, a.y) : 0.f;
    }
    // per channel: bias, then the taps in order 0..8 (one FMA each)
    float acc[Co];
#pragma unroll
    for (int c = 0; c < Co; ++c) acc[c] = bs[c];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const float4 *w4 = reinterpret_cast<const float4 *>(ws + r * Co);
#pragma unroll
        for (int c4 = 0; c4 < Co / 4; ++c4) {
            const float4 q = w4[c4];
            acc[4 * c4 + 0] = fmaf(q.x, v[r], acc[4 * c4 + 0]);
            acc[4 * c4 + 1] = fmaf(q.y, v[r], acc[4 * c4 + 1]);
            acc[4 * c4 + 2] = fmaf(q.z, v[r], acc[4 * c4 + 2]);
            acc[4 * c4 + 3] = fmaf(q.w, v[r], acc[4 * c4 + 3]);
        }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(y + n * Co);
#pragma unroll
    for (int c8 = 0; c8 < Co / 8; ++c8) {
        uint32_t h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 8 * c8 + 2 * j;
            const __nv_bfloat162 t = __floats2bfloat162_rn(fmaxf(acc[c], 0.f), fmaxf(acc[c + 1], 0.f));
            h[j] = *reinterpret_cast<const uint32_t *>(&t);
        }
        dst[c8] = make_uint4(h[0], h[1], h[2], h[3]);
    }
}

// weights [Co][Ci][9] FP32 -> [Co][Kp] BF16 in the order k = r Ci + ci (r = ky * 3 + kx), zero padded
__global__ void k_cnn_weights_bf16(const float *__restrict__ w, int Co, int Ci, int Kp,
                                   __nv_bfloat16 *__restrict__ out) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)Co * Kp) return;
    const int co = (int)(i / Kp), k = (int)(i - (long)co * Kp);
    float v = 0.f;
    if (k < 9 * Ci) {
        const int r = k / Ci, ci = k - r * Ci;
        v = w[((long)co * Ci + ci) * 9 + r];
    }
    out[i] = __float2bfloat16_rn(v);
}

// mean over the Q positions of NHWC activations [B][Q][C]: pool[b][c]
__global__ void k_cnn_pool_nhwc(const float *__restrict__ a, int B, int C, int Q, float *__restrict__ pool) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * C) return;
    const int b = i / C, c = i - b * C;
    float s = 0.f;
    for (int p = 0; p < Q; ++p) s += a[((long)b * Q + p) * C + c];
    pool[i] = s / Q;
}

// gradient into the last conv output: g[b][c][p] = gpool[b][c] / Q where a > 0
__global__ void k_cnn_pool_back(const float *__restrict__ gpool, const float *__restrict__ a, int BC, int Q,
                                float *__restrict__ g) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)BC * Q) return;
    g[i] = a[i] > 0.f ? gpool[i / Q] / Q : 0.f;
}

// bias gradient, per block row y: dbp[y][c] = sum over its share of b < B, p < Q
// of g[b][c][p] (fixed order); the rows are summed in order afterwards
__global__ void k_cnn_bias_grad(const float *__restrict__ g, int B, int C, int Q, float *__restrict__ dbp) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (long i = (long)blockIdx.y * blockDim.x + threadIdx.x; i < (long)B * Q; i += (long)gridDim.y * blockDim.x) {
        const long b = i / Q, p = i - b * Q;
        s += g[(b * C + c) * Q + p];
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float r[32];
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += r[w];
        dbp[(long)blockIdx.y * C + c] = t;
    }
}

// ------------------------------------------------------------- heads
struct M3 { double a[9]; };   // row-major 3 x 3

__device__ __forceinline__ void cross(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// columns b1, b2, b3 of the Gram-Schmidt rotation of (a1, a2); also returns
// the norms |a1| and |u| (u = a2 - (b1.a2) b1) and b1.a2
__device__ void gs(const float *a, double *b1, double *b2, double *b3, double *n1, double *n2, double *d) {
    double a1[3] = {a[0], a[1], a[2]}, a2[3] = {a[3], a[4], a[5]}, u[3];
    *n1 = sqrt(dot(a1, a1));
    for (int i = 0; i < 3; ++i) b1[i] = a1[i] / *n1;
    *d = dot(b1, a2);
    for (int i = 0; i < 3; ++i) u[i] = a2[i] - *d * b1[i];
    *n2 = sqrt(dot(u, u));
    for (int i = 0; i < 3; ++i) b2[i] = u[i] / *n2;
    cross(b1, b2, b3);
}

// the projector's matrix of a unit quaternion (w, x, y, z)
__device__ M3 quat_matrix(const double *q) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    return {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
             2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
             2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
}

// cubic operator s (0..23): the s-th signed permutation matrix of determinant
// +1 in the order (permutation, sign bits) enumerated below
__device__ M3 cubic_op(int s) {
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int parity[6] = {1, -1, -1, 1, 1, -1};
    int n = 0;
    for (int p = 0; p < 6; ++p)
        for (int sg = 0; sg < 8; ++sg) {
            const int signs = ((sg & 1) ? -1 : 1) * ((sg & 2) ? -1 : 1) * ((sg & 4) ? -1 : 1);
            if (signs * parity[p] != 1) continue;
            if (n++ != s) continue;
            M3 m = {{0, 0, 0, 0, 0, 0, 0, 0, 0}};
            for (int r = 0; r < 3; ++r) m.a[r * 3 + perms[p][r]] = ((sg >> r) & 1) ? -1.0 : 1.0;
            return m;
        }
    return {{1, 0, 0, 0, 1, 0, 0, 0, 1}};
}

// one thread per pattern: winner-takes-all loss over heads and cubic operators
__global__ void k_cnn_head_loss(const float *__restrict__ out, int B, int k, const double *__restrict__ qgt,
                                float *__restrict__ gout, double *__restrict__ loss_sum, int *__restrict__ winners) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double my = 0.0;
    if (b < B) {
        const M3 Rg = quat_matrix(qgt + 4 * b);
        double best = 1e300;
        int bh = 0, bs = 0;
        for (int h = 0; h < k; ++h) {
            double b1[3], b2[3], b3[3], n1, n2, d;
            gs(out + ((long)b * k + h) * 6, b1, b2, b3, &n1, &n2, &d);
            for (int s = 0; s < 24; ++s) {
                const M3 S = cubic_op(s);
                double l = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        const double t = S.a[i * 3] * Rg.a[j] + S.a[i * 3 + 1] * Rg.a[3 + j] + S.a[i * 3 + 2] * Rg.a[6 + j];
                        const double r = j == 0 ? b1[i] : (j == 1 ? b2[i] : b3[i]);
                        l += (r - t) * (r - t);
                    }
                if (l < best) {
                    best = l;
                    bh = h;
                    bs = s;
                }
            }
        }
        my = best / B;
        if (winners) {
            winners[2 * b] = bh;
            winners[2 * b + 1] = bs;
        }
        // gradient of |R - S Rg|^2 through Gram-Schmidt, scaled by 1/B
        double b1[3], b2[3], b3[3], n1, n2, d;
        const float *a = out + ((long)b * k + bh) * 6;
        gs(a, b1, b2, b3, &n1, &n2, &d);
        const M3 S = cubic_op(bs);
        double g1[3], g2[3], g3[3];
        for (int i = 0; i < 3; ++i) {
            double t[3];
            for (int j = 0; j < 3; ++j)
                t[j] = S.a[i * 3] * Rg.a[j] + S.a[i * 3 + 1] * Rg.a[3 + j] + S.a[i * 3 + 2] * Rg.a[6 + j];
            g1[i] = 2.0 * (b1[i] - t[0]) / B;
            g2[i] = 2.0 * (b2[i] - t[1]) / B;
            g3[i] = 2.0 * (b3[i] - t[2]) / B;
        }
        double gb1[3], gb2[3], t[3], gu[3], ga1[3], ga2[3];
        cross(b2, g3, t);
        for (int i = 0; i < 3; ++i) gb1[i] = g1[i] + t[i];
        cross(g3, b1, t);
        for (int i = 0; i < 3; ++i) gb2[i] = g2[i] + t[i];
        const double pb2 = dot(b2, gb2);
        for (int i = 0; i < 3; ++i) gu[i] = (gb2[i] - pb2 * b2[i]) / n2;
        const double pu = dot(b1, gu);
        for (int i = 0; i < 3; ++i) {
            ga2[i] = gu[i] - pu * b1[i];
            gb1[i] += -pu * a[3 + i] - d * gu[i];
        }
        const double pb1 = dot(b1, gb1);
        for (int i = 0; i < 3; ++i) ga1[i] = (gb1[i] - pb1 * b1[i]) / n1;
        for (int h = 0; h < k; ++h)
            for (int i = 0; i < 6; ++i) {
                double v = 0.0;
                if (h == bh) v = i < 3 ? ga1[i] : ga2[i - 3];
                gout[((long)b * k + h) * 6 + i] = (float)v;
            }
    }
    for (int o = 16; o; o >>= 1) my += __shfl_xor_sync(0xffffffffu, my, o);
    if ((threadIdx.x & 31) == 0 && loss_sum) atomicAdd(loss_sum, my);
}

// proposals: quaternion (w >= 0) of the Gram-Schmidt rotation of every head
__global__ void k_cnn_proposals(const float *__restrict__ out, int n, double *__restrict__ quats) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double b1[3], b2[3], b3[3], n1, n2, d;
    gs(out + (long)i * 6, b1, b2, b3, &n1, &n2, &d);
    // R has columns b1, b2, b3: R[r][c]
    const double R[9] = {b1[0], b2[0], b3[0], b1[1], b2[1], b3[1], b1[2], b2[2], b3[2]};
    // Shepperd: the largest of 4w^2, 4x^2, 4y^2, 4z^2 decides the branch
    const double t = R[0] + R[4] + R[8];
    const double c[4] = {1 + t, 1 + R[0] - R[4] - R[8], 1 - R[0] + R[4] - R[8], 1 - R[0] - R[4] + R[8]};
    int m = 0;
    for (int j = 1; j < 4; ++j)
        if (c[j] > c[m]) m = j;
    const double s = 2.0 * sqrt(c[m]);
    double w, x, y, z;
    if (m == 0) {
        w = s / 4; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
    } else if (m == 1) {
        x = s / 4; w = (R[7] - R[5]) / s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
    } else if (m == 2) {
        y = s / 4; w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; z = (R[5] + R[7]) / s;
    } else {
        z = s / 4; w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s;
    }
    double nn = sqrt(w * w + x * x + y * y + z * z);
    if (w < 0) nn = -nn;
    double *q = quats + 4L * i;
    q[0] = w / nn;
    q[1] = x / nn;
    q[2] = y / nn;
    q[3] = z / nn;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// proposal h of every pattern: q[p] = prop[p][h]
__global__ void k_take_head(const double *__restrict__ prop, int P, int k, int h, double *__restrict__ q) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    for (int i = 0; i < 4; ++i) q[4 * p + i] = prop[((long)p * k + h) * 4 + i];
}

// keep the proposal with the highest correlation peak (ties: lowest head)
__global__ void k_keep_best(const float *__restrict__ peak_h, const double *__restrict__ q_h, int P, int h,
                            float *__restrict__ best_peak, double *__restrict__ best_q, int *__restrict__ best_h) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    if (h == 0 || peak_h[p] > best_peak[p]) {
        best_peak[p] = peak_h[p];
        if (best_h) best_h[p] = h;
        for (int i = 0; i < 4; ++i) best_q[4 * p + i] = q_h[4 * p + i];
    }
}

// fallback flags: refined peak below tau on a non-degenerate pattern; count them
__global__ void k_fallback_flags(const float *__restrict__ peak, const int *__restrict__ degen, int P, float tau,
                                 int *__restrict__ fb, int *__restrict__ count) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (p < P) {
        f = (!degen[p] && !(peak[p] >= tau)) ? 1 : 0;
        fb[p] = f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, __popc(m));
}

// search mask (patterns without fallback are skipped as if degenerate) and
// the seeds of the second refinement: library orientation of the best
// template where a fallback happens, the current orientation elsewhere
__global__ void k_fallback_mask(const int *__restrict__ degen, const int *__restrict__ fb, int P,
                                int *__restrict__ mask) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) mask[p] = degen[p] || !fb[p];
}
__global__ void k_fallback_seeds(const int *__restrict__ fb, const int *__restrict__ best,
                                 const double *__restrict__ lib_q, const double *__restrict__ cur, int P,
                                 double *__restrict__ seeds) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const bool use = fb[p] && best[p] >= 0;
    for (int i = 0; i < 4; ++i) seeds[4 * p + i] = use ? lib_q[4L * best[p] + i] : cur[4 * p + i];
}

// the fallback batch by pattern pairs (one block of 1024 threads): every
// pair (2j, 2j + 1) with a flagged member, in order, at (2i, 2i + 1), so that
// each pattern keeps the partner it shares a complex inverse transform with
// in the pair-peak kernels; flag_c marks the flagged members (a last pair
// without a second pattern repeats the first, unflagged); pairs[0] = count
__global__ void __launch_bounds__(1024) k_fallback_list(const int *__restrict__ fb, int P, int *__restrict__ idx,
                                                        int *__restrict__ flag_c, int *__restrict__ pairs) {
    __shared__ int sums[1024];
    const int U = (P + 1) / 2;
    const int t = threadIdx.x, per = (U + 1023) / 1024, b = t * per, e = min(U, b + per);
    auto flagged = [&](int j) { return fb[2 * j] != 0 || (2 * j + 1 < P && fb[2 * j + 1] != 0); };
    int c = 0;
    for (int j = b; j < e; ++j) c += flagged(j) ? 1 : 0;
    sums[t] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan of the counts
        const int v = t >= o ? sums[t - o] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int pos = sums[t] - c;
    for (int j = b; j < e; ++j) {
        if (!flagged(j)) continue;
        const bool two = 2 * j + 1 < P;
        idx[2 * pos] = 2 * j;
        flag_c[2 * pos] = fb[2 * j] != 0;
        idx[2 * pos + 1] = two ? 2 * j + 1 : 2 * j;
        flag_c[2 * pos + 1] = two && fb[2 * j + 1] != 0;
        ++pos;
    }
    if (t == 1023) pairs[0] = sums[1023];
}
// row i of dst = row idx[i] of src (rows of len elements)
template <class T>
__global__ void k_gather_rows(const T *__restrict__ src, size_t len, const int *__restrict__ idx, int n,
                              T *__restrict__ dst) {
    const size_t total = (size_t)n * len;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / len;
        dst[i] = src[(size_t)idx[r] * len + (i - r * len)];
    }
}
// seeds of the listed patterns: for flagged ones the library orientation of
// the best template, else (and where there is none) the current orientation
__global__ void k_fallback_seeds_list(const int *__restrict__ idx, const int *__restrict__ flag_c,
                                      const int *__restrict__ best, const double *__restrict__ lib_q,
                                      const double *__restrict__ cur, int n, double *__restrict__ seeds) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *src = flag_c[i] && best[i] >= 0 ? lib_q + 4L * best[i] : cur + 4L * idx[i];
    for (int k = 0; k < 4; ++k) seeds[4 * i + k] = src[k];
}
// the flagged patterns' results back to their own slots
__global__ void k_fallback_scatter(const int *__restrict__ idx, const int *__restrict__ flag_c, int n,
                                   const double *__restrict__ q_c, const float *__restrict__ peak_c,
                                   const int *__restrict__ it_c, double *__restrict__ q, float *__restrict__ peak,
                                   int *__restrict__ iters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag_c[i]) return;
    const int p = idx[i];
    for (int k = 0; k < 4; ++k) q[4L * p + k] = q_c[4 * i + k];
    peak[p] = peak_c[i];
    iters[p] = it_c[i];
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {
const int kCh[6] = {1, 32, 64, 64, 128, 128};
constexpr int kHidden = 256;
}

long cnn_num_params(int k) {
    long n = 0;
    for (int l = 0; l < 5; ++l) n += (long)kCh[l + 1] * kCh[l] * 9 + kCh[l + 1];
    return n + (long)kHidden * kCh[5] + kHidden + 6L * k * kHidden + 6L * k;
}

size_t cnn_act_floats(int B, int k) {
    size_t n = 0;
    int s = 128;
    for (int l = 0; l < 5; ++l) {
        s /= 2;
        n += (size_t)B * kCh[l + 1] * s * s;
    }
    return n + (size_t)B * (kCh[5] + kHidden + 6 * k) + 2 * (size_t)B;   // pool, h1, out, affine
}

// split partials of one weight gradient, and per-block bias partials
constexpr size_t kPartFloats = (size_t)1 << 22;
constexpr int kBiasRows = 64;
constexpr size_t kBiasPartFloats = (size_t)kBiasRows * 512;

size_t cnn_grad_floats(int B, int k) {
    return 2 * (size_t)B * kCh[1] * 64 * 64 + (size_t)B * (kCh[5] + kHidden + 6 * k) + kPartFloats + kBiasPartFloats;
}

namespace {
struct Layout {
    long cw[5], cb[5], f1w, f1b, f2w, f2b;
    explicit Layout(int k) {
        long o = 0;
        for (int l = 0; l < 5; ++l) {
            cw[l] = o;
            o += (long)kCh[l + 1] * kCh[l] * 9;
            cb[l] = o;
            o += kCh[l + 1];
        }
        f1w = o;
        o += (long)kHidden * kCh[5];
        f1b = o;
        o += kHidden;
        f2w = o;
        o += 6L * k * kHidden;
        f2b = o;
    }
};
struct Acts {
    float *a[5], *pool, *h1, *out;
    float2 *affine;
    Acts(float *base, int B, int k) {
        int s = 128;
        for (int l = 0; l < 5; ++l) {
            s /= 2;
            a[l] = base;
            base += (size_t)B * kCh[l + 1] * s * s;
        }
        pool = base;
        base += (size_t)B * kCh[5];
        h1 = base;
        base += (size_t)B * kHidden;
        out = base;
        base += (size_t)B * 6 * k;
        affine = reinterpret_cast<float2 *>(base);
    }
};
#define CNN_TRY(x)                              \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)
}  // namespace

cudaError_t launch_cnn_forward(const float *params, int k, const CnnInput &in, int B, float *act, int *launches,
                               cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const Layout L(k);
    Acts A(act, B, k);
    k_cnn_stats<<<B, 256, 0, st>>>(in.x, in.img_stride, in.row_stride, in.ox, in.oy, 128, A.affine);
    CNN_TRY(cudaGetLastError());
    int n_launch = 1;
    int s = 128;
    for (int l = 0; l < 5; ++l) {
        const int so = s / 2;
        Src src = l == 0 ? Src{in.x, 1, 128, in.img_stride, in.row_stride, in.ox, in.oy, A.affine}
                         : Src{A.a[l - 1], kCh[l], s, (long)kCh[l] * s * s, s, 0, 0, nullptr};
        CNN_TRY(gemm(kCh[l + 1], B * so * so, kCh[l] * 9, 1, LoadW{params + L.cw[l], kCh[l] * 9},
                     LoadIm2col{src, so}, EpConv{A.a[l], params + L.cb[l], kCh[l + 1], so * so}, st));
        ++n_launch;
        s = so;
    }
    k_cnn_pool<<<(B * kCh[5] + 255) / 256, 256, 0, st>>>(A.a[4], B * kCh[5], 16, A.pool);
    CNN_TRY(cudaGetLastError());
    CNN_TRY(gemm(kHidden, B, kCh[5], 1, LoadW{params + L.f1w, kCh[5]}, LoadRows{A.pool, kCh[5]},
                 EpVec{A.h1, params + L.f1b, kHidden, true}, st));
    CNN_TRY(gemm(6 * k, B, kHidden, 1, LoadW{params + L.f2w, kHidden}, LoadRows{A.h1, kHidden},
                 EpVec{A.out, params + L.f2b, 6 * k, false}, st));
    if (launches) *launches += n_launch + 3;
    return cudaSuccess;
}

namespace {
constexpr int kBf16Kp[5] = {0, 320, 576, 576, 1152};   // 9 Ci rounded up to a multiple of 64
size_t bf16_weight_elems() {
    size_t n = 0;
    for (int l = 1; l < 5; ++l) n += (size_t)kCh[l + 1] * kBf16Kp[l];
    return n;
}
}  // namespace

size_t cnn_bf16_work_bytes(int) { return 2 * bf16_weight_elems() + 256; }

cudaError_t launch_cnn_forward_bf16(const float *params, int k, const CnnInput &in, int B, float *act, void *work,
                                    int *err, int num_sms, int *launches, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const Layout L(k);
    Acts A(act, B, k);   // a[0..3] hold BF16 NHWC activations, a[4] FP32 NHWC
    __nv_bfloat16 *wl = static_cast<__nv_bfloat16 *>(work);
    k_cnn_stats<<<B, 256, 0, st>>>(in.x, in.img_stride, in.row_stride, in.ox, in.oy, 128, A.affine);
    CNN_TRY(cudaGetLastError());
    int n_launch = 1;
    {
        const long np = (long)B * 64 * 64;
        k_cnn_conv1_nhwc<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
            in.x, in.img_stride, in.row_stride, in.ox, in.oy, A.affine, params + L.cw[0], params + L.cb[0], B,
            reinterpret_cast<__nv_bfloat16 *>(A.a[0]));
        CNN_TRY(cudaGetLastError());
        ++n_launch;
    }
    for (int l = 1; l < 5; ++l) {
        const int Kp = kBf16Kp[l], Co = kCh[l + 1];
        const long nw = (long)Co * Kp;
        k_cnn_weights_bf16<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(params + L.cw[l], Co, kCh[l], Kp, wl);
        CNN_TRY(cudaGetLastError());
        CNN_TRY(launch_conv_tc(l, A.a[l - 1], B, wl, params + L.cb[l], A.a[l], err, num_sms, st));
        n_launch += 2;
        wl += nw;
    }
    k_cnn_pool_nhwc<<<(B * kCh[5] + 255) / 256, 256, 0, st>>>(A.a[4], B, kCh[5], 16, A.pool);
    CNN_TRY(cudaGetLastError());
    CNN_TRY(gemm(kHidden, B, kCh[5], 1, LoadW{params + L.f1w, kCh[5]}, LoadRows{A.pool, kCh[5]},
                 EpVec{A.h1, params + L.f1b, kHidden, true}, st));
    CNN_TRY(gemm(6 * k, B, kHidden, 1, LoadW{params + L.f2w, kHidden}, LoadRows{A.h1, kHidden},
                 EpVec{A.out, params + L.f2b, 6 * k, false}, st));
    if (launches) *launches += n_launch + 3;
    return cudaSuccess;
}

const float *cnn_output(float *act, int B, int k) { return Acts(act, B, k).out; }

cudaError_t launch_cnn_backward(const float *params, int k, const CnnInput &in, int B, float *act, float *gbuf,
                                const double *qgt, double *loss_sum, int *winners, float *grad, int num_sms,
                                int *launches, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const Layout L(k);
    Acts A(act, B, k);
    const size_t big = (size_t)B * kCh[1] * 64 * 64;
    float *gbufs[2] = {gbuf, gbuf + big};
    float *gout = gbuf + 2 * big, *gh1 = gout + (size_t)B * 6 * k, *gpool = gh1 + (size_t)B * kHidden;
    float *part = gpool + (size_t)B * kCh[5], *bpart = part + kPartFloats;
    int n_launch = 0;
    // weight gradient out[M][N] = A^T B over the batch, reduced over K in splits
    // whose partials are summed in a fixed order (no atomics: reproducible)
    auto weight_grad = [&](int M, int N, int K, auto la, auto lb, float *out) -> cudaError_t {
        int splits = grad_splits(M, N, K, num_sms);
        while (splits > 1 && (size_t)splits * M * N > kPartFloats) splits = (splits + 1) / 2;
        const int kper = split_kper(K, splits);
        splits = (K + kper - 1) / kper;
        cudaError_t e = gemm_kper(M, N, K, kper, la, lb, EpPartial{part, M, N}, st);
        if (e != cudaSuccess) return e;
        const long n = (long)M * N;
        k_sum_partials<<<(unsigned)min((n + 255) / 256, 4096L), 256, 0, st>>>(part, splits, n, out);
        n_launch += 2;
        return cudaGetLastError();
    };
    auto bias_grad = [&](const float *g, int C, int Q, int rows, float *db) -> cudaError_t {
        rows = max(1, min(rows, kBiasRows));
        k_cnn_bias_grad<<<dim3(C, rows), 256, 0, st>>>(g, B, C, Q, bpart);
        k_sum_partials<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(bpart, rows, C, db);
        n_launch += 2;
        return cudaGetLastError();
    };
    CNN_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * cnn_num_params(k), st));
    k_cnn_head_loss<<<(B + 127) / 128, 128, 0, st>>>(A.out, B, k, qgt, gout, loss_sum, winners);
    CNN_TRY(cudaGetLastError());
    // fc2: dW2 = gout^T h1, db2, gh1 = (W2^T gout) where h1 > 0
    const int M2 = 6 * k;
    CNN_TRY(weight_grad(M2, kHidden, B, LoadRowsT{gout, M2}, LoadRowsB{A.h1, kHidden}, grad + L.f2w));
    CNN_TRY(bias_grad(gout, M2, 1, 1, grad + L.f2b));
    CNN_TRY(gemm(kHidden, B, M2, 1, LoadWT{params + L.f2w, kHidden}, LoadRows{gout, M2},
                 EpMasked{gh1, A.h1, kHidden}, st));
    // fc1: dW1 = gh1^T pool, db1, gpool = W1^T gh1
    CNN_TRY(weight_grad(kHidden, kCh[5], B, LoadRowsT{gh1, kHidden}, LoadRowsB{A.pool, kCh[5]}, grad + L.f1w));
    CNN_TRY(bias_grad(gh1, kHidden, 1, 1, grad + L.f1b));
    CNN_TRY(gemm(kCh[5], B, kHidden, 1, LoadWT{params + L.f1w, kCh[5]}, LoadRows{gh1, kHidden},
                 EpStore{gpool, kCh[5]}, st));
    n_launch += 3;
    // mean pool, then the conv layers from the last to the first
    int so = 4, cur = 0;
    {
        const long n = (long)B * kCh[5] * 16;
        k_cnn_pool_back<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gpool, A.a[4], B * kCh[5], 16, gbufs[cur]);
        CNN_TRY(cudaGetLastError());
        ++n_launch;
    }
    for (int l = 4; l >= 0; --l) {
        const int si = 2 * so, ci = kCh[l], co = kCh[l + 1];
        const float *g = gbufs[cur];
        Src src = l == 0 ? Src{in.x, 1, 128, in.img_stride, in.row_stride, in.ox, in.oy, A.affine}
                         : Src{A.a[l - 1], ci, si, (long)ci * si * si, si, 0, 0, nullptr};
        CNN_TRY(weight_grad(co, ci * 9, B * so * so, LoadGradT{g, co, so * so}, LoadIm2colT{src, so},
                            grad + L.cw[l]));
        CNN_TRY(bias_grad(g, co, so * so, 2 * num_sms / co, grad + L.cb[l]));
        if (l > 0) {   // gradient into the previous layer's output, through its ReLU
            CNN_TRY(gemm(ci, B * si * si, co * 9, 1, LoadWconvT{params + L.cw[l], ci}, LoadGradScatter{g, co, so},
                         EpMaskedImg{gbufs[cur ^ 1], A.a[l - 1], ci, si * si}, st));
            ++n_launch;
            cur ^= 1;
        }
        so = si;
    }
    if (launches) *launches += n_launch;
    return cudaSuccess;
}

cudaError_t launch_cnn_proposals(const float *out, int n_heads_total, double *quats, cudaStream_t st) {
    if (n_heads_total <= 0) return cudaSuccess;
    k_cnn_proposals<<<(n_heads_total + 127) / 128, 128, 0, st>>>(out, n_heads_total, quats);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, long n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t st) {
    const float c1 = (float)(1.0 - pow((double)b1, t)), c2 = (float)(1.0 - pow((double)b2, t));
    k_adam<<<1024, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_take_head(const double *prop, int P, int k, int h, double *q, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_take_head<<<(P + 255) / 256, 256, 0, st>>>(prop, P, k, h, q);
    return cudaGetLastError();
}

cudaError_t launch_keep_best(const float *peak_h, const double *q_h, int P, int h, float *best_peak, double *best_q,
                             int *best_h, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_keep_best<<<(P + 255) / 256, 256, 0, st>>>(peak_h, q_h, P, h, best_peak, best_q, best_h);
    return cudaGetLastError();
}

cudaError_t launch_fallback_flags(const float *peak, const int *degen, int P, float tau, int *fb, int *count,
                                  cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_fallback_flags<<<(P + 255) / 256, 256, 0, st>>>(peak, degen, P, tau, fb, count);
    return cudaGetLastError();
}

cudaError_t launch_fallback_mask(const int *degen, const int *fb, int P, int *mask, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_fallback_mask<<<(P + 255) / 256, 256, 0, st>>>(degen, fb, P, mask);
    return cudaGetLastError();
}

cudaError_t launch_fallback_list(const int *fb, int P, int *idx, int *flag_c, int *pairs, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_fallback_list<<<1, 1024, 0, st>>>(fb, P, idx, flag_c, pairs);
    return cudaGetLastError();
}

template <class T>
static cudaError_t gather_rows(const T *src, size_t len, const int *idx, int n, T *dst, cudaStream_t st) {
    if (n <= 0 || len == 0) return cudaSuccess;
    const size_t total = (size_t)n * len;
    const int blocks = (int)((total + 255) / 256 < 65536 ? (total + 255) / 256 : 65536);
    k_gather_rows<T><<<blocks, 256, 0, st>>>(src, len, idx, n, dst);
    return cudaGetLastError();
}
cudaError_t launch_gather_rows(const float *src, size_t len, const int *idx, int n, float *dst, cudaStream_t st) {
    return gather_rows(src, len, idx, n, dst, st);
}
cudaError_t launch_gather_rows(const double *src, size_t len, const int *idx, int n, double *dst, cudaStream_t st) {
    return gather_rows(src, len, idx, n, dst, st);
}

cudaError_t launch_fallback_seeds_list(const int *idx, const int *flag_c, const int *best, const double *lib_q,
                                       const double *cur, int n, double *seeds, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_fallback_seeds_list<<<(n + 255) / 256, 256, 0, st>>>(idx, flag_c, best, lib_q, cur, n, seeds);
    return cudaGetLastError();
}

cudaError_t launch_fallback_scatter(const int *idx, const int *flag_c, int n, const double *q_c, const float *peak_c,
                                    const int *it_c, double *q, float *peak, int *iters, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_fallback_scatter<<<(n + 255) / 256, 256, 0, st>>>(idx, flag_c, n, q_c, peak_c, it_c, q, peak, iters);
    return cudaGetLastError();
}

cudaError_t launch_fallback_seeds(const int *fb, const int *best, const double *lib_q, const double *cur, int P,
                                  double *seeds, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_fallback_seeds<<<(P + 255) / 256, 256, 0, st>>>(fb, best, lib_q, cur, P, seeds);
    return cudaGetLastError();
}
