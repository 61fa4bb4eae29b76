// Pre-processing, the all-sides search kernel and the single-surface peak
// kernel for N in {16, 32, 64, 128}: each CTA holds one N x N complex array in
// shared memory (rows padded to N + 1) and transforms it with a radix-2 FFT
// whose butterflies are spread over the lanes of a warp.
//
// Paper: FFT section (Eq. 4 transform, filtering, windowing, normalisation by
// the autocorrelations), Eqs. 3 and 6 (correlation surface), peak up-sampling.
#include "common.cuh"
#include "generic.cuh"
#include "kernels.cuh"

namespace {

using namespace gen;

// --------------------------------------------------------------------------
// pre-processing: crop, standardise, window, FFT, band-pass, unit norm
// --------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_prep(const float *__restrict__ img, PrepArgs a,
                                                   float2 *__restrict__ spec,
                                                   float *__restrict__ spatial,
                                                   int *__restrict__ degen,
                                                   const int *__restrict__ active) {
    constexpr int LD = N + 1, HW = N / 2 + 1;
    if (active && !active[blockIdx.x]) return;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *twf = buf + N * LD;
    float2 *twi = twf + N / 2;
    __shared__ double red[33];
    const int p = blockIdx.x, tid = threadIdx.x;
    const float *src = img + (size_t)p * a.W * a.H;
    float2 *out = spec + (size_t)p * N * HW;

    make_twiddles<N>(twf, -1);
    make_twiddles<N>(twi, +1);
    double s = 0.0;
    for (int idx = tid; idx < N * N; idx += kThreads) {
        int r = idx / N, c = idx % N;
        float v = src[(size_t)(a.oy + r) * a.W + a.ox + c];
        buf[r * LD + c] = make_float2(v, 0.f);
        s += v;
    }
    const double mean = block_sum(s, red) / (N * N);
    double ss = 0.0;
    for (int idx = tid; idx < N * N; idx += kThreads) {
        double d = buf[(idx / N) * LD + idx % N].x - mean;
        ss += d * d;
    }
    const double sd = sqrt(block_sum(ss, red) / (N * N));
    bool bad = !(sd > 1e-12 * (1.0 + fabs(mean)));
    double energy = 0.0;
    if (!bad) {
        const float m = (float)mean, inv = (float)(1.0 / sd);
        for (int idx = tid; idx < N * N; idx += kThreads) {
            int r = idx / N, c = idx % N;
            float wr = a.window ? 0.5f * (1.f - cospif(2.f * r / N)) : 1.f;
            float wc = a.window ? 0.5f * (1.f - cospif(2.f * c / N)) : 1.f;
            float v = buf[r * LD + c].x;
            buf[r * LD + c] = make_float2((v - m) * inv * wr * wc, 0.f);
        }
        __syncthreads();
        fft2_smem<N>(buf, twf);
        double e = 0.0;
        for (int idx = tid; idx < N * N; idx += kThreads) {
            int u = idx / N, v = idx % N;
            float fu = (float)(u < N / 2 ? u : u - N), fv = (float)(v < N / 2 ? v : v - N);
            float rho2 = fu * fu + fv * fv;
            float h = -expm1f(-rho2 * a.inv2shp) * expf(-rho2 * a.inv2slp);
            float2 X = buf[u * LD + v];
            X = make_float2(X.x * h, X.y * h);
            buf[u * LD + v] = X;
            e += (double)X.x * X.x + (double)X.y * X.y;
        }
        energy = block_sum(e, red);
        bad = !(energy > 0.0);
    }
    if (tid == 0 && degen) degen[p] = bad ? 1 : 0;
    if (bad) {
        for (int idx = tid; idx < N * HW; idx += kThreads) out[idx] = make_float2(0.f, 0.f);
        if (spatial)
            for (int idx = tid; idx < N * N; idx += kThreads) spatial[(size_t)p * N * N + idx] = 0.f;
        return;
    }
    const float sc = (float)(1.0 / sqrt(energy));
    for (int idx = tid; idx < N * HW; idx += kThreads) {
        int u = idx / HW, v = idx % HW;
        float2 X = buf[u * LD + v];
        out[idx] = make_float2(X.x * sc, X.y * sc);
    }
    if (spatial) {
        __syncthreads();
        for (int idx = tid; idx < N * N; idx += kThreads) {
            int u = idx / N, v = idx % N;
            float2 X = buf[u * LD + v];
            buf[u * LD + v] = make_float2(X.x * sc, X.y * sc);
        }
        __syncthreads();
        fft2_smem<N>(buf, twi);
        const float invn = 1.f / N;
        for (int idx = tid; idx < N * N; idx += kThreads)
            spatial[(size_t)p * N * N + idx] = buf[(idx / N) * LD + idx % N].x * invn;
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_search_generic(const float2 *__restrict__ St, int T,
                                                             const float2 *__restrict__ Sp,
                                                             const int *__restrict__ degen,
                                                             int pairs_per_cta,
                                                             unsigned long long *__restrict__ keys,
                                                             float *__restrict__ peaks_all,
                                                             const int *__restrict__ cand, int kc) {
    const int p = blockIdx.y;
    if (degen[p]) return;
    const int npairs = ((cand ? kc : T) + 1) / 2;
    const int pb = blockIdx.x * pairs_per_cta, pe = min(npairs, pb + pairs_per_cta);
    search_body<N>(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc);
}

__device__ __forceinline__ float parabola(float cm, float c0, float cp) {
    float den = cm - 2.f * c0 + cp;
    if (!(den < 0.f)) return 0.f;
    float d = (cm - cp) / (2.f * den);
    return fminf(0.5f, fmaxf(-0.5f, d));
}

// --------------------------------------------------------------------------
// one surface per pattern: integer argmax (ties -> lowest row-major shift),
// peak value and parabolic sub-pixel shift
// --------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_pair_peak(const float2 *__restrict__ St,
                                                        const int *__restrict__ tidx,
                                                        const float2 *__restrict__ Sp,
                                                        const int *__restrict__ degen,
                                                        const int *__restrict__ active,
                                                        float *__restrict__ peak,
                                                        float *__restrict__ shift) {
    constexpr int LD = N + 1, HW = N / 2 + 1;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *twi = buf + N * LD;
    __shared__ float rv[kThreads / 32];
    __shared__ int ri[kThreads / 32];
    __shared__ int s_best;
    const int p = blockIdx.x;
    if (active && !active[p]) return;
    const int t = tidx ? tidx[p] : p;
    if ((degen && degen[p]) || t < 0) {
        if (threadIdx.x == 0) {
            peak[p] = 0.f;
            shift[2 * p] = 0.f;
            shift[2 * p + 1] = 0.f;
        }
        return;
    }
    make_twiddles<N>(twi, +1);
    const float2 *st = St + (size_t)t * N * HW;
    build_pair_spectrum<N>(buf, st, st, Sp + (size_t)p * N * HW);
    __syncthreads();
    fft2_smem<N>(buf, twi);
    // the imaginary part of Z = X + i X is a copy of the surface; use the real part
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int idx = threadIdx.x; idx < N * N; idx += kThreads) {
        float v = buf[(idx / N) * LD + idx % N].x;
        if (v > bv) { bv = v; bi = idx; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { rv[w] = bv; ri[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k)
            if (rv[k] > bv || (rv[k] == bv && ri[k] < bi)) { bv = rv[k]; bi = ri[k]; }
        s_best = bi;
        const int y0 = bi / N, x0 = bi % N;
        const float c0 = buf[y0 * LD + x0].x;
        const float cxm = buf[y0 * LD + ((x0 + N - 1) & (N - 1))].x;
        const float cxp = buf[y0 * LD + ((x0 + 1) & (N - 1))].x;
        const float cym = buf[((y0 + N - 1) & (N - 1)) * LD + x0].x;
        const float cyp = buf[((y0 + 1) & (N - 1)) * LD + x0].x;
        peak[p] = c0;
        shift[2 * p] = (float)(x0 < N / 2 ? x0 : x0 - N) + parabola(cxm, c0, cxp);
        shift[2 * p + 1] = (float)(y0 < N / 2 ? y0 : y0 - N) + parabola(cym, c0, cyp);
    }
}

__global__ void k_keys_to_best(const unsigned long long *__restrict__ keys, int P, int *__restrict__ best) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    unsigned long long k = keys[p];
    best[p] = k ? (int)(0xffffffffu - (uint32_t)(k & 0xffffffffull)) : -1;
}

template <int N>
size_t smem_bytes_generic() { return sizeof(float2) * ((size_t)N * (N + 1) + N); }

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N>
cudaError_t prep_n(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                   const int *active, cudaStream_t st) {
    size_t sm = smem_bytes_generic<N>();
    cudaError_t e = set_smem(k_prep<N>, sm);
    if (e != cudaSuccess) return e;
    k_prep<N><<<P, kThreads, sm, st>>>(img, a, spec, spatial, degen, active);
    return cudaGetLastError();
}

template <int N>
cudaError_t search_n(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                     unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st,
                     const int *cand = nullptr, int kc = 0) {
    size_t sm = smem_bytes_generic<N>();
    cudaError_t e = set_smem(k_search_generic<N>, sm);
    if (e != cudaSuccess) return e;
    const int npairs = ((cand ? kc : T) + 1) / 2;
    // enough CTAs to fill the GPU a few times over, at least 4 pairs each
    long want = (long)num_sms * 8;
    int chunks = (int)((want + P - 1) / P);
    chunks = max(1, min(chunks, (npairs + 3) / 4));
    int ppc = (npairs + chunks - 1) / chunks;
    chunks = (npairs + ppc - 1) / ppc;
    dim3 grid(chunks, P);
    k_search_generic<N><<<grid, kThreads, sm, st>>>(St, T, Sp, degen, ppc, keys, peaks_all, cand, kc);
    return cudaGetLastError();
}

template <int N>
cudaError_t pair_peak_n(const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                        const int *active, int P, float *peak, float *shift, cudaStream_t st) {
    size_t sm = smem_bytes_generic<N>();
    cudaError_t e = set_smem(k_pair_peak<N>, sm);
    if (e != cudaSuccess) return e;
    k_pair_peak<N><<<P, kThreads, sm, st>>>(St, tidx, Sp, degen, active, peak, shift);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_search128(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                             unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st);

cudaError_t launch_prep(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial,
                        int *degen, const int *active, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    switch (a.N) {
        case 16: return prep_n<16>(img, P, a, spec, spatial, degen, active, st);
        case 32: return prep_n<32>(img, P, a, spec, spatial, degen, active, st);
        case 64: return prep_n<64>(img, P, a, spec, spatial, degen, active, st);
        case 128: return prep_n<128>(img, P, a, spec, spatial, degen, active, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_search(int N, const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                          unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st) {
    if (P <= 0 || T <= 0) return cudaSuccess;
    switch (N) {
        case 16: return search_n<16>(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
        case 32: return search_n<32>(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
        case 64: return search_n<64>(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
        case 128: return launch_search128(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_search_generic128(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                                     unsigned long long *keys, float *peaks_all, int num_sms,
                                     cudaStream_t st) {
    return search_n<128>(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
}

cudaError_t launch_search_list(int N, const float2 *St, const int *cand, int kc, const float2 *Sp,
                               const int *degen, int P, unsigned long long *keys, float *peaks, int num_sms,
                               cudaStream_t st) {
    if (P <= 0 || kc <= 0) return cudaSuccess;
    switch (N) {
        case 16: return search_n<16>(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
        case 32: return search_n<32>(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
        case 64: return search_n<64>(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
        case 128: return search_n<128>(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pair_peak(int N, const float2 *St, const int *tidx, const float2 *Sp,
                             const int *degen, const int *active, int P, float *peak, float *shift,
                             cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    switch (N) {
        case 16: return pair_peak_n<16>(St, tidx, Sp, degen, active, P, peak, shift, st);
        case 32: return pair_peak_n<32>(St, tidx, Sp, degen, active, P, peak, shift, st);
        case 64: return pair_peak_n<64>(St, tidx, Sp, degen, active, P, peak, shift, st);
        case 128: return pair_peak_n<128>(St, tidx, Sp, degen, active, P, peak, shift, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_keys_to_best(const unsigned long long *keys, int P, int *best, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_keys_to_best<<<(P + 255) / 256, 256, 0, st>>>(keys, P, best);
    return cudaGetLastError();
}
