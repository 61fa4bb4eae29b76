// Pre-processing, the all-sides search kernel and the single-surface peak
// kernel for N in {16, 32, 64, 128}.  The search and peak kernels hold one
// N x N complex array in shared memory (rows padded to N + 1) and transform it
// with a radix-2 FFT whose butterflies are spread over the lanes of a warp;
// the pre-processing transforms real images at half that work (below).
//
// Paper: FFT section (Eq. 4 transform, filtering, windowing, normalisation by
// the autocorrelations), Eqs. 3 and 6 (correlation surface), peak up-sampling.
#include "common.cuh"
#include "generic.cuh"
#include "kernels.cuh"

namespace {

using namespace gen;

// --------------------------------------------------------------------------
// pre-processing of real images with half the transform work: image rows
// 2r and 2r+1 form one complex line (rows transformed as N/2 complex lines,
// then split by Hermitian symmetry into R[y][0..N/2]); the columns of R are
// transformed as their even- and odd-row halves (N/2-point transforms) joined
// by one radix-2 stage.  Bins 0 and N/2 of every row are real, so they share
// one complex slot per row pair.  The N/2 x (N+1) complex array (66 KB at
// N = 128) lets three CTAs share an SM.  The spatial output runs the same
// steps backwards.
// layout of buf after the row split, row pr (image rows 2pr, 2pr+1):
//   [0]        (Ra[0], Ra[N/2])   real bins of row 2pr
//   [1, N/2)   Ra[v]
//   [N/2]      (Rb[0], Rb[N/2])   real bins of row 2pr+1
//   (N/2, N)   Rb[v - N/2]
// after the column transforms, S[u][v] (1 <= v < N/2) is at buf[u][v] for
// u < N/2 and at buf[u - N/2][N/2 + v] above; columns 0 and N/2 go to c0, cH.
// --------------------------------------------------------------------------
template <int N>
constexpr size_t smem_prep_real() {
    return sizeof(float2) * ((size_t)(N / 2) * (N + 1) + N + N / 2 + 2 * N);
}

// threads per CTA: more warps for the larger sides hide the shared-memory and
// global-load latency of the line transforms
template <int N>
constexpr int prep_threads() { return N >= 128 ? 512 : kThreads; }
template <int N>
constexpr int peak_threads() { return N >= 128 ? 1024 : kThreads; }

template <int N, int PT = prep_threads<N>()>
__global__ void __launch_bounds__(PT) k_prep_real(const float *__restrict__ img, PrepArgs a,
                                                        float2 *__restrict__ spec, float *__restrict__ spatial,
                                                        int *__restrict__ degen, const int *__restrict__ active) {
    constexpr int H = N / 2, LD = N + 1, HW = N / 2 + 1;
    if (active && !active[blockIdx.x]) return;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);   // [H][LD]
    float2 *twN = buf + H * LD;                            // e^{-2 pi i k / N},   k < N/2
    float2 *twNi = twN + N / 2;                            // e^{+2 pi i k / N}
    float2 *twH = twNi + N / 2;                            // e^{-2 pi i k / (N/2)}, k < N/4
    float2 *twHi = twH + N / 4;
    float2 *c0 = twHi + N / 4;                             // S[u][0],   u < N
    float2 *cH = c0 + N;                                   // S[u][N/2], u < N
    __shared__ double red[33];
    const int p = blockIdx.x, tid = threadIdx.x;
    const float *src = img + (size_t)p * a.W * a.H;
    float2 *out = spec + (size_t)p * N * HW;
    make_twiddles<N>(twN, -1);
    make_twiddles<N>(twNi, +1);
    make_twiddles<H>(twH, -1);
    make_twiddles<H>(twHi, +1);
    // ---- load (rows 2pr, 2pr+1 into the real and imaginary parts of buf row pr) and statistics:
    // one pass of FP32 sums of (x - x0), x0 the crop's first pixel (a constant crop has exactly
    // zero variance; the shift keeps the per-thread sums well conditioned), combined in FP64
    const float x0 = __ldg(src + (size_t)a.oy * a.W + a.ox);
    float s1 = 0.f, s2 = 0.f;
    for (int idx = tid; idx < N * N; idx += PT) {
        const int r = idx / N, c = idx % N;
        const float v = src[(size_t)(a.oy + r) * a.W + a.ox + c];
        reinterpret_cast<float *>(buf + (r >> 1) * LD + c)[r & 1] = v;
        const float d = v - x0;
        s1 += d;
        s2 = fmaf(d, d, s2);
    }
    const double m1 = block_sum_f(s1, red) / (N * N), m2 = block_sum_f(s2, red) / (N * N);
    const double mean = x0 + m1, var = m2 - m1 * m1;
    const double sd = var > 0.0 ? sqrt(var) : 0.0;
    bool bad = !(sd > 1e-12 * (1.0 + fabs(mean)));
    double energy = 0.0;
    if (!bad) {
        const float m = (float)mean, inv = (float)(1.0 / sd);
        for (int idx = tid; idx < H * N; idx += PT) {
            const int pr = idx / N, c = idx % N;
            const float wc = (a.window ? 0.5f * (1.f - cospif(2.f * c / N)) : 1.f) * inv;
            const float w0 = a.window ? 0.5f * (1.f - cospif(2.f * (2 * pr) / N)) : 1.f;
            const float w1 = a.window ? 0.5f * (1.f - cospif(2.f * (2 * pr + 1) / N)) : 1.f;
            const float2 z = buf[pr * LD + c];
            buf[pr * LD + c] = make_float2((z.x - m) * wc * w0, (z.y - m) * wc * w1);
        }
        __syncthreads();
        smem_fft_lines<N>(buf, H, LD, 1, twN);   // rows
        __syncthreads();
        {   // split every packed row into its two real rows' half spectra
            constexpr int ITEMS = H * (N / 2), PER = (ITEMS + PT - 1) / PT;
            float2 ra[PER], rb[PER];
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int it = tid + k * PT;
                if (it < ITEMS) {
                    const int pr = it / (N / 2), v = it % (N / 2);
                    const float2 *row = buf + pr * LD;
                    if (v == 0) {
                        const float2 z0 = row[0], zh = row[N / 2];
                        ra[k] = make_float2(z0.x, zh.x);
                        rb[k] = make_float2(z0.y, zh.y);
                    } else {
                        const float2 zv = row[v], zn = row[N - v];
                        ra[k] = make_float2(0.5f * (zv.x + zn.x), 0.5f * (zv.y - zn.y));
                        rb[k] = make_float2(0.5f * (zv.y + zn.y), 0.5f * (zn.x - zv.x));
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int it = tid + k * PT;
                if (it < ITEMS) {
                    const int pr = it / (N / 2), v = it % (N / 2);
                    buf[pr * LD + v] = ra[k];
                    buf[pr * LD + N / 2 + v] = rb[k];
                }
            }
        }
        __syncthreads();
        smem_fft_lines<H>(buf, N, 1, LD, twH);   // even-row and odd-row halves of every column
        __syncthreads();
        // join the halves: X[u] = E[u] + w^u O[u], X[u + N/2] = E[u] - w^u O[u]
        for (int it = tid; it < H * (N / 2); it += PT) {
            const int u = it / (N / 2), v = it % (N / 2);
            const float2 w = twN[u];
            if (v == 0) {
                // columns 0 and N/2: the packed real sequences, split first
                const int un = (H - u) & (H - 1);
                const float2 we = buf[u * LD], wen = buf[un * LD];
                const float2 wo = buf[u * LD + N / 2], won = buf[un * LD + N / 2];
                const float2 ae = make_float2(0.5f * (we.x + wen.x), 0.5f * (we.y - wen.y));
                const float2 be = make_float2(0.5f * (we.y + wen.y), 0.5f * (wen.x - we.x));
                const float2 ao = c_mul(make_float2(0.5f * (wo.x + won.x), 0.5f * (wo.y - won.y)), w);
                const float2 bo = c_mul(make_float2(0.5f * (wo.y + won.y), 0.5f * (won.x - wo.x)), w);
                c0[u] = c_add(ae, ao);
                c0[u + H] = c_sub(ae, ao);
                cH[u] = c_add(be, bo);
                cH[u + H] = c_sub(be, bo);
            } else {
                const float2 e = buf[u * LD + v], o = c_mul(buf[u * LD + N / 2 + v], w);
                buf[u * LD + v] = c_add(e, o);
                buf[u * LD + N / 2 + v] = c_sub(e, o);
            }
        }
        __syncthreads();
        // band-pass and the filtered energy (bins 1..N/2-1 stand for their mirror images too)
        float e = 0.f;
        for (int it = tid; it < N * HW; it += PT) {
            const int u = it / HW, v = it % HW;
            float2 *x = v == 0 ? c0 + u : (v == N / 2 ? cH + u : buf + (u & (H - 1)) * LD + (u >= H ? N / 2 : 0) + v);
            const float fu = (float)(u < N / 2 ? u : u - N), fv = (float)(v < N / 2 ? v : v - N);
            const float rho2 = fu * fu + fv * fv;
            const float h = -expm1f(-rho2 * a.inv2shp) * expf(-rho2 * a.inv2slp);
            const float2 X = make_float2(x->x * h, x->y * h);
            *x = X;
            e = fmaf(v == 0 || v == N / 2 ? 1.f : 2.f, X.x * X.x + X.y * X.y, e);
        }
        energy = block_sum_f(e, red);
        bad = !(energy > 0.0);
    }
    if (tid == 0 && degen) degen[p] = bad ? 1 : 0;
    if (bad) {
        for (int idx = tid; idx < N * HW; idx += PT) out[idx] = make_float2(0.f, 0.f);
        if (spatial)
            for (int idx = tid; idx < N * N; idx += PT) spatial[(size_t)p * N * N + idx] = 0.f;
        return;
    }
    const float sc = (float)(1.0 / sqrt(energy));
    for (int it = tid; it < N * HW; it += PT) {
        const int u = it / HW, v = it % HW;
        const float2 X = v == 0 ? c0[u] : (v == N / 2 ? cH[u] : buf[(u & (H - 1)) * LD + (u >= H ? N / 2 : 0) + v]);
        out[it] = make_float2(X.x * sc, X.y * sc);
    }
    if (!spatial) return;
    __syncthreads();
    // ---- spatial image: undo the join (E = X[u] + X[u + N/2], O = w^-u (X[u] - X[u + N/2]))
    for (int it = tid; it < H * (N / 2); it += PT) {
        const int u = it / (N / 2), v = it % (N / 2);
        const float2 wi = twNi[u];
        if (v == 0) {
            const float2 e0 = c_add(c0[u], c0[u + H]), o0 = c_mul(c_sub(c0[u], c0[u + H]), wi);
            const float2 eh = c_add(cH[u], cH[u + H]), oh = c_mul(c_sub(cH[u], cH[u + H]), wi);
            // pack the two real-output columns: E0 + i EH, O0 + i OH (scaled)
            buf[u * LD] = make_float2(sc * (e0.x - eh.y), sc * (e0.y + eh.x));
            buf[u * LD + N / 2] = make_float2(sc * (o0.x - oh.y), sc * (o0.y + oh.x));
        } else {
            const float2 x0 = buf[u * LD + v], x1 = buf[u * LD + N / 2 + v];
            const float2 e = c_add(x0, x1), o = c_mul(c_sub(x0, x1), wi);
            buf[u * LD + v] = make_float2(e.x * sc, e.y * sc);
            buf[u * LD + N / 2 + v] = make_float2(o.x * sc, o.y * sc);
        }
    }
    __syncthreads();
    smem_fft_lines<H>(buf, N, 1, LD, twHi);   // columns back: R'[y][v] in the split layout
    __syncthreads();
    {   // rows 2pr, 2pr+1 as one complex line: z[v] = Ra[v] + i Rb[v], conjugate-symmetric extension
        constexpr int ITEMS = H * N, PER = (ITEMS + PT - 1) / PT;
        float2 zz[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int it = tid + k * PT;
            if (it < ITEMS) {
                const int pr = it / N, v = it % N;
                const float2 *row = buf + pr * LD;
                const int w = v <= N / 2 ? v : N - v;
                float2 ra, rb;
                if (w == 0 || w == N / 2) {
                    ra = make_float2(w == 0 ? row[0].x : row[0].y, 0.f);
                    rb = make_float2(w == 0 ? row[N / 2].x : row[N / 2].y, 0.f);
                } else {
                    ra = row[w];
                    rb = row[N / 2 + w];
                    if (v > N / 2) {
                        ra.y = -ra.y;
                        rb.y = -rb.y;
                    }
                }
                zz[k] = make_float2(ra.x - rb.y, ra.y + rb.x);
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int it = tid + k * PT;
            if (it < ITEMS) buf[(it / N) * LD + it % N] = zz[k];
        }
    }
    __syncthreads();
    smem_fft_lines<N>(buf, H, LD, 1, twNi);   // rows back
    __syncthreads();
    const float invn = 1.f / N;
    for (int idx = tid; idx < N * N; idx += PT) {
        const int r = idx / N, c = idx % N;
        const float2 z = buf[(r >> 1) * LD + c];
        spatial[(size_t)p * N * N + idx] = ((r & 1) ? z.y : z.x) * invn;
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
// Two patterns per CTA: Z = X_a + i X_b with X_s = conj(S_t(s)) S_p(s), so the
// real and imaginary parts of one complex inverse transform are the two
// surfaces.  A pattern that is skipped (inactive) or has no template
// contributes X = 0.
template <int N, int QT = peak_threads<N>()>
__global__ void __launch_bounds__(QT) k_pair_peak(const float2 *__restrict__ St,
                                                        const int *__restrict__ tidx,
                                                        const float2 *__restrict__ Sp,
                                                        const int *__restrict__ degen,
                                                        const int *__restrict__ active, int P,
                                                        float *__restrict__ peak,
                                                        float *__restrict__ shift, int *__restrict__ argmax) {
    constexpr int LD = N + 1, HW = N / 2 + 1;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *twi = buf + N * LD;
    __shared__ float rv[2][QT / 32];
    __shared__ int ri[2][QT / 32];
    const int tid = threadIdx.x;
    int pp[2], mode[2], tt[2];   // mode: 0 skip, 1 zero outputs, 2 compute
    for (int s = 0; s < 2; ++s) {
        pp[s] = 2 * blockIdx.x + s;
        const int p = pp[s];
        if (p >= P || (active && !active[p])) {
            mode[s] = 0;
            tt[s] = 0;
            continue;
        }
        tt[s] = tidx ? tidx[p] : p;
        mode[s] = ((degen && degen[p]) || tt[s] < 0) ? 1 : 2;
        if (mode[s] == 1 && tid == 0) {
            peak[p] = 0.f;
            shift[2 * p] = 0.f;
            shift[2 * p + 1] = 0.f;
        }
    }
    if (mode[0] != 2 && mode[1] != 2) return;
    make_twiddles<N>(twi, +1);
    const float2 *ta = St + (size_t)(mode[0] == 2 ? tt[0] : 0) * N * HW;
    const float2 *tb = St + (size_t)(mode[1] == 2 ? tt[1] : 0) * N * HW;
    const float2 *qa = Sp + (size_t)(mode[0] == 2 ? pp[0] : 0) * N * HW;
    const float2 *qb = Sp + (size_t)(mode[1] == 2 ? pp[1] : 0) * N * HW;
    const float fa = mode[0] == 2 ? 1.f : 0.f, fb = mode[1] == 2 ? 1.f : 0.f;
    for (int idx = tid; idx < N * N; idx += QT) {
        const int r = idx / N, c = idx % N;
        const bool direct = c <= N / 2;
        const int k = direct ? r * HW + c : ((N - r) & (N - 1)) * HW + (N - c);   // conj(X(-u, -v)) above N/2
        float2 x1 = c_mulcj(ta[k], qa[k]), x2 = c_mulcj(tb[k], qb[k]);
        x1 = make_float2(x1.x * fa, x1.y * fa);
        x2 = make_float2(x2.x * fb, x2.y * fb);
        buf[r * LD + c] = direct ? make_float2(x1.x - x2.y, x1.y + x2.x) : make_float2(x1.x + x2.y, -x1.y + x2.x);
    }
    __syncthreads();
    fft2_smem<N>(buf, twi);
    float bv[2] = {-INFINITY, -INFINITY};
    int bi[2] = {0x7fffffff, 0x7fffffff};
    for (int idx = tid; idx < N * N; idx += QT) {
        const float2 v = buf[(idx / N) * LD + idx % N];
        if (v.x > bv[0]) { bv[0] = v.x; bi[0] = idx; }
        if (v.y > bv[1]) { bv[1] = v.y; bi[1] = idx; }
    }
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv[s], o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi[s], o);
            if (ov > bv[s] || (ov == bv[s] && oi < bi[s])) { bv[s] = ov; bi[s] = oi; }
        }
        if (lane == 0) { rv[s][w] = bv[s]; ri[s][w] = bi[s]; }
    }
    __syncthreads();
    if (tid < 2 && mode[tid] == 2) {
        const int s = tid, p = pp[s];
        float b = rv[s][0];
        int i0 = ri[s][0];
        for (int k = 1; k < QT / 32; ++k)
            if (rv[s][k] > b || (rv[s][k] == b && ri[s][k] < i0)) { b = rv[s][k]; i0 = ri[s][k]; }
        const int y0 = i0 / N, x0 = i0 % N;
        auto at = [&](int y, int x) {
            const float2 z = buf[y * LD + x];
            return s ? z.y : z.x;
        };
        const float c0 = at(y0, x0);
        const float cxm = at(y0, (x0 + N - 1) & (N - 1)), cxp = at(y0, (x0 + 1) & (N - 1));
        const float cym = at((y0 + N - 1) & (N - 1), x0), cyp = at((y0 + 1) & (N - 1), x0);
        peak[p] = c0;
        shift[2 * p] = (float)(x0 < N / 2 ? x0 : x0 - N) + parabola(cxm, c0, cxp);
        shift[2 * p + 1] = (float)(y0 < N / 2 ? y0 : y0 - N) + parabola(cym, c0, cyp);
        if (argmax) argmax[p] = i0;
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
    const size_t sm = smem_prep_real<N>();
    cudaError_t e = set_smem(k_prep_real<N>, sm);
    if (e != cudaSuccess) return e;
    k_prep_real<N><<<P, prep_threads<N>(), sm, st>>>(img, a, spec, spatial, degen, active);
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
                        const int *active, int P, float *peak, float *shift, int *argmax, cudaStream_t st) {
    size_t sm = smem_bytes_generic<N>();
    cudaError_t e = set_smem(k_pair_peak<N>, sm);
    if (e != cudaSuccess) return e;
    k_pair_peak<N><<<(P + 1) / 2, peak_threads<N>(), sm, st>>>(St, tidx, Sp, degen, active, P, peak, shift, argmax);
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
                             cudaStream_t st, int *argmax) {
    if (P <= 0) return cudaSuccess;
    switch (N) {
        case 16: return pair_peak_n<16>(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        case 32: return pair_peak_n<32>(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        case 64: return pair_peak_n<64>(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        case 128: return pair_peak_n<128>(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_keys_to_best(const unsigned long long *keys, int P, int *best, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_keys_to_best<<<(P + 255) / 256, 256, 0, st>>>(keys, P, best);
    return cudaGetLastError();
}
