// Pre-processing, all-pairs search and single-surface peak for detectors
// too large for one SM's shared memory (N = 256: a complex N x N array is
// 512 KB).  Each CTA owns an N x N complex work array in global memory (it
// stays in L2: the grid is persistent, about two CTAs per SM) and transforms
// it line by line: rows by one warp each, columns in tiles of 8 adjacent
// columns staged through shared memory (coalesced).
//
// Paper: FFT section (Eq. 4, filtering, windowing, normalisation), Eqs. 3
// and 6 (correlation surface), peak up-sampling (parabolic reading).
#include "big.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace {

using namespace bigk;

// --------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads) k_prep_big(const float *__restrict__ img, int P, PrepArgs a,
                                                       float2 *__restrict__ spec, float *__restrict__ spatial,
                                                       int *__restrict__ degen, const int *__restrict__ active,
                                                       float2 *__restrict__ work) {
    constexpr int HW = N / 2 + 1;
    extern __shared__ float4 smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float2 *tw = sm + (size_t)N * kColTile;
    __shared__ double red[33];
    float2 *Z = work + (size_t)blockIdx.x * N * N;
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        if (active && !active[p]) continue;
        const float *src = img + (size_t)p * a.W * a.H;
        float2 *out = spec + (size_t)p * N * HW;
        double s = 0.0;
        for (int i = threadIdx.x; i < N * N; i += kThreads)
            s += src[(size_t)(a.oy + i / N) * a.W + a.ox + i % N];
        const double mean = block_sum_b(s, red) / ((double)N * N);
        double ss = 0.0;
        for (int i = threadIdx.x; i < N * N; i += kThreads) {
            const double d = src[(size_t)(a.oy + i / N) * a.W + a.ox + i % N] - mean;
            ss += d * d;
        }
        const double sd = sqrt(block_sum_b(ss, red) / ((double)N * N));
        bool bad = !(sd > 1e-12 * (1.0 + fabs(mean)));
        double energy = 0.0;
        if (!bad) {
            make_tw<N>(tw, -1);
            const float m = (float)mean, inv = (float)(1.0 / sd);
            for (int i = threadIdx.x; i < N * N; i += kThreads) {
                const int r = i / N, c = i % N;
                const float wr = a.window ? 0.5f * (1.f - cospif(2.f * r / N)) : 1.f;
                const float wc = a.window ? 0.5f * (1.f - cospif(2.f * c / N)) : 1.f;
                const float v = src[(size_t)(a.oy + r) * a.W + a.ox + c];
                Z[i] = make_float2((v - m) * inv * wr * wc, 0.f);
            }
            __syncthreads();
            fft2_global<N>(Z, sm, tw);
            double e = 0.0;
            for (int i = threadIdx.x; i < N * N; i += kThreads) {
                const int u = i / N, v = i % N;
                const float fu = (float)(u < N / 2 ? u : u - N), fv = (float)(v < N / 2 ? v : v - N);
                const float rho2 = fu * fu + fv * fv;
                const float h = -expm1f(-rho2 * a.inv2shp) * expf(-rho2 * a.inv2slp);
                float2 X = Z[i];
                X = make_float2(X.x * h, X.y * h);
                Z[i] = X;
                e += (double)X.x * X.x + (double)X.y * X.y;
            }
            energy = block_sum_b(e, red);
            bad = !(energy > 0.0);
        }
        if (threadIdx.x == 0 && degen) degen[p] = bad ? 1 : 0;
        if (bad) {
            for (int i = threadIdx.x; i < N * HW; i += kThreads) out[i] = make_float2(0.f, 0.f);
            if (spatial)
                for (int i = threadIdx.x; i < N * N; i += kThreads) spatial[(size_t)p * N * N + i] = 0.f;
            __syncthreads();
            continue;
        }
        const float sc = (float)(1.0 / sqrt(energy));
        for (int i = threadIdx.x; i < N * HW; i += kThreads) {
            const float2 X = Z[(size_t)(i / HW) * N + i % HW];
            out[i] = make_float2(X.x * sc, X.y * sc);
        }
        if (spatial) {
            for (int i = threadIdx.x; i < N * N; i += kThreads) {
                const float2 X = Z[i];
                Z[i] = make_float2(X.x * sc, X.y * sc);
            }
            make_tw<N>(tw, +1);
            __syncthreads();
            fft2_global<N>(Z, sm, tw);
            const float invn = 1.f / N;
            for (int i = threadIdx.x; i < N * N; i += kThreads) spatial[(size_t)p * N * N + i] = Z[i].x * invn;
        }
        __syncthreads();
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_search_big(const float2 *__restrict__ St, int T,
                                                         const float2 *__restrict__ Sp,
                                                         const int *__restrict__ degen, int P, int ppc,
                                                         unsigned long long *__restrict__ keys,
                                                         float *__restrict__ peaks_all,
                                                         float2 *__restrict__ work,
                                                         const int *__restrict__ cand, int kc) {
    extern __shared__ float4 smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float2 *tw = sm + (size_t)N * kColTile;
    __shared__ float redf[33];
    float2 *Z = work + (size_t)blockIdx.x * N * N;
    make_tw<N>(tw, +1);
    __syncthreads();
    // slots: every template, or each pattern's candidate list (entries < 0 are empty)
    const int n = cand ? kc : T;
    const int npairs = (n + 1) / 2, nchunks = (npairs + ppc - 1) / ppc;
    for (long item = blockIdx.x; item < (long)P * nchunks; item += gridDim.x) {
        const int p = (int)(item / nchunks), ch = (int)(item % nchunks);
        if (degen[p]) continue;
        search_body<N>(St, T, Sp, p, ch * ppc, min(npairs, (ch + 1) * ppc), keys, peaks_all, Z, sm, tw, redf, cand,
                       kc);
    }
}

__device__ __forceinline__ float parabola_b(float cm, float c0, float cp) {
    const float den = cm - 2.f * c0 + cp;
    if (!(den < 0.f)) return 0.f;
    const float d = (cm - cp) / (2.f * den);
    return fminf(0.5f, fmaxf(-0.5f, d));
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_pair_peak_big(const float2 *__restrict__ St,
                                                            const int *__restrict__ tidx,
                                                            const float2 *__restrict__ Sp,
                                                            const int *__restrict__ degen,
                                                            const int *__restrict__ active, int P,
                                                            float *__restrict__ peak, float *__restrict__ shift,
                                                            float2 *__restrict__ work) {
    constexpr int HW = N / 2 + 1;
    extern __shared__ float4 smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float2 *tw = sm + (size_t)N * kColTile;
    __shared__ float rv[kWarps];
    __shared__ int ri[kWarps];
    float2 *Z = work + (size_t)blockIdx.x * N * N;
    make_tw<N>(tw, +1);
    __syncthreads();
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        if (active && !active[p]) continue;
        const int t = tidx ? tidx[p] : p;
        if ((degen && degen[p]) || t < 0) {
            if (threadIdx.x == 0) { peak[p] = 0.f; shift[2 * p] = 0.f; shift[2 * p + 1] = 0.f; }
            continue;
        }
        const float2 *st = St + (size_t)t * N * HW;
        build_pair_big<N>(Z, st, st, Sp + (size_t)p * N * HW);
        __syncthreads();
        fft2_global<N>(Z, sm, tw);
        float bv = -INFINITY;
        int bi = 0x7fffffff;
        for (int i = threadIdx.x; i < N * N; i += kThreads) {
            const float v = Z[i].x;
            if (v > bv) { bv = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) { rv[w] = bv; ri[w] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < kWarps; ++k)
                if (rv[k] > bv || (rv[k] == bv && ri[k] < bi)) { bv = rv[k]; bi = ri[k]; }
            const int y0 = bi / N, x0 = bi % N;
            const float c0 = Z[bi].x;
            const float cxm = Z[(size_t)y0 * N + ((x0 + N - 1) & (N - 1))].x;
            const float cxp = Z[(size_t)y0 * N + ((x0 + 1) & (N - 1))].x;
            const float cym = Z[(size_t)((y0 + N - 1) & (N - 1)) * N + x0].x;
            const float cyp = Z[(size_t)((y0 + 1) & (N - 1)) * N + x0].x;
            peak[p] = c0;
            shift[2 * p] = (float)(x0 < N / 2 ? x0 : x0 - N) + parabola_b(cxm, c0, cxp);
            shift[2 * p + 1] = (float)(y0 < N / 2 ? y0 : y0 - N) + parabola_b(cym, c0, cyp);
        }
        __syncthreads();
    }
}

template <typename K>
cudaError_t set_smem_b(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int big_grid(int num_sms, long items) {
    long g = 2L * (num_sms > 0 ? num_sms : 1);
    return (int)(items < g ? (items > 0 ? items : 1) : g);
}

size_t big_work_bytes(int N, int grid) { return sizeof(float2) * (size_t)N * N * grid; }

cudaError_t launch_prep_big(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                            const int *active, float2 *work, int grid, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (a.N != 256) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_b(k_prep_big<256>, smem_big(256));
    if (e != cudaSuccess) return e;
    k_prep_big<256><<<grid, kThreads, smem_big(256), st>>>(img, P, a, spec, spatial, degen, active, work);
    return cudaGetLastError();
}

cudaError_t launch_search_big(int N, const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                              unsigned long long *keys, float *peaks_all, float2 *work, int grid,
                              cudaStream_t st, const int *cand, int kc) {
    if (P <= 0 || (cand ? kc : T) <= 0) return cudaSuccess;
    if (N != 256) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_b(k_search_big<256>, smem_big(256));
    if (e != cudaSuccess) return e;
    const int npairs = ((cand ? kc : T) + 1) / 2;
    // chunks of pairs so that there are at least ~4 work items per CTA
    long want = 4L * grid;
    int nchunks = (int)((want + P - 1) / P);
    nchunks = nchunks < 1 ? 1 : (nchunks > npairs ? npairs : nchunks);
    const int ppc = (npairs + nchunks - 1) / nchunks;
    k_search_big<256><<<grid, kThreads, smem_big(256), st>>>(St, T, Sp, degen, P, ppc, keys, peaks_all, work,
                                                             cand, kc);
    return cudaGetLastError();
}

cudaError_t launch_pair_peak_big(int N, const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                 const int *active, int P, float *peak, float *shift, float2 *work, int grid,
                                 cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (N != 256) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_b(k_pair_peak_big<256>, smem_big(256));
    if (e != cudaSuccess) return e;
    k_pair_peak_big<256><<<grid, kThreads, smem_big(256), st>>>(St, tidx, Sp, degen, active, P, peak, shift, work);
    return cudaGetLastError();
}
