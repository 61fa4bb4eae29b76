// The native 200 x 200 detector side: pre-processing, the all-pairs search
// and the single-surface peak.
//
// Paper: FFT section (Eq. 4 transform, window, band-pass, normalisation by the
// autocorrelations; footnote 1: the crop to 2^n only makes the transform and
// the filters easier, so a 200 px detector can be used whole), Eqs. 3 and 6
// (the correlation surface), the peak fit of Fig. 1 C.
//
// The complex 200 x 200 array of two packed surfaces (320 KB) fits no SM, so
// one template is correlated at a time through the real-output inverse
// transform, whose working array is the 200 x 101 half spectrum (162 KB, in
// shared memory): X = conj(S_t) S_p over the stored half (u < 200, v <= 100);
// the 101 columns are inverse-transformed over u (200 points); each row y
// then goes back to 200 real values through one 100-point complex transform,
// z[k] = E[k] + i O[k] with E[k] = C[k] + conj C[100 - k] and O[k] =
// (C[k] - conj C[100 - k]) e^{+2 pi i k / 200}, whose real and imaginary
// parts are the even and odd columns of the surface.  The pre-processing runs
// the same steps forwards (rows as 100-point transforms of (x[2n], x[2n+1])
// split into the 101-point half row, then the columns) and, for the filtered
// image, backwards.
//
// Line transforms: one warp per line, Stockham autosort passes in shared
// memory between two per-warp line buffers, radices 8, 5, 5 (200 points) and
// 4, 5, 5 (100 points), the small DFTs in registers, the twiddles from one
// table of e^{+2 pi i e / 200}.
#include "common.cuh"
#include "generic.cuh"
#include "kernels.cuh"

namespace {

constexpr int N = 200, HW = N / 2 + 1, M = N / 2, NT = 512, NWARP = NT / 32;
// shared memory (float2 units): the half spectrum [N][HW], two line buffers
// per warp, the twiddle table
constexpr int OFF_SCR = N * HW;
constexpr int OFF_TW = OFF_SCR + NWARP * 2 * N;
constexpr int SMEM_F2 = OFF_TW + N;
constexpr size_t SMEM_BYTES = sizeof(float2) * SMEM_F2;   // 214,400 B

// e^{SIGN 2 pi i e / 200} from the table of e^{+2 pi i e / 200}
template <int SIGN>
__device__ __forceinline__ float2 tw_at(const float2 *tw, int e) {
    const float2 w = tw[e];
    return SIGN > 0 ? w : make_float2(w.x, -w.y);
}

// small DFTs in registers, V[p] = sum_q v[q] e^{SIGN 2 pi i p q / R}, natural order
template <int SIGN>
__device__ __forceinline__ void dft4(float2 (&v)[4]) {
    const float2 s02 = c_add(v[0], v[2]), d02 = c_sub(v[0], v[2]);
    const float2 s13 = c_add(v[1], v[3]);
    const float2 d13 = SIGN > 0 ? c_mul_pi(c_sub(v[1], v[3])) : c_mul_mi(c_sub(v[1], v[3]));
    v[0] = c_add(s02, s13);
    v[2] = c_sub(s02, s13);
    v[1] = c_add(d02, d13);
    v[3] = c_sub(d02, d13);
}
// radix 5 from the sums and differences of the conjugate-symmetric pairs
// (v1, v4) and (v2, v3): V_1,4 = v0 + c1 t1 + c2 t2 +- i SIGN (s1 t3 + s2 t4),
// V_2,3 = v0 + c2 t1 + c1 t2 +- i SIGN (s2 t3 - s1 t4)
template <int SIGN>
__device__ __forceinline__ void dft5(float2 (&v)[5]) {
    constexpr float c1 = Tw<1, 5, +1>::re, s1 = Tw<1, 5, +1>::im;
    constexpr float c2 = Tw<2, 5, +1>::re, s2 = Tw<2, 5, +1>::im;
    const float2 t1 = c_add(v[1], v[4]), t2 = c_add(v[2], v[3]);
    const float2 t3 = c_sub(v[1], v[4]), t4 = c_sub(v[2], v[3]);
    const float2 a1 = make_float2(fmaf(c1, t1.x, fmaf(c2, t2.x, v[0].x)), fmaf(c1, t1.y, fmaf(c2, t2.y, v[0].y)));
    const float2 a2 = make_float2(fmaf(c2, t1.x, fmaf(c1, t2.x, v[0].x)), fmaf(c2, t1.y, fmaf(c1, t2.y, v[0].y)));
    float2 b1 = make_float2(fmaf(s1, t3.x, s2 * t4.x), fmaf(s1, t3.y, s2 * t4.y));
    float2 b2 = make_float2(fmaf(s2, t3.x, -s1 * t4.x), fmaf(s2, t3.y, -s1 * t4.y));
    // i SIGN b
    b1 = SIGN > 0 ? c_mul_pi(b1) : c_mul_mi(b1);
    b2 = SIGN > 0 ? c_mul_pi(b2) : c_mul_mi(b2);
    v[0] = c_add(v[0], c_add(t1, t2));
    v[1] = c_add(a1, b1);
    v[4] = c_sub(a1, b1);
    v[2] = c_add(a2, b2);
    v[3] = c_sub(a2, b2);
}
template <int SIGN>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    fft_reg_dif<8, SIGN>(v);   // v[p] = V[bitrev3(p)]
    const float2 t1 = v[1], t3 = v[3], t4 = v[4], t6 = v[6];
    v[1] = t4;   // V1 was at 4
    v[4] = t1;   // V4 was at 1
    v[3] = t6;   // V3 was at 6
    v[6] = t3;   // V6 was at 3
}
template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    if constexpr (R == 4) dft4<SIGN>(v);
    else if constexpr (R == 5) dft5<SIGN>(v);
    else dft8<SIGN>(v);
}

// one Stockham pass of radix R over a line of L points (x -> y), sub-transform
// length Ns before the pass: task j (k = j mod Ns) reads x[j + q L/R],
// multiplies by e^{SIGN 2 pi i q k / (Ns R)}, takes the R-point DFT and writes
// y[(j / Ns) Ns R + k + p Ns]
template <int R, int SIGN>
__device__ __forceinline__ void stockham(const float2 *__restrict__ x, float2 *__restrict__ y, int L, int Ns,
                                         const float2 *tw, int lane) {
    const int m = L / R, step = N / (Ns * R);
    for (int j = lane; j < m; j += 32) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = x[j + q * m];
        if (k) {
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = c_mul(v[q], tw_at<SIGN>(tw, q * k * step));
        }
        dft<R, SIGN>(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int p = 0; p < R; ++p) y[base + p * Ns] = v[p];
    }
    __syncwarp();
}
// 200-point line: a (natural order) -> b (natural order); a is overwritten
template <int SIGN>
__device__ __forceinline__ void line200(float2 *a, float2 *b, const float2 *tw, int lane) {
    stockham<8, SIGN>(a, b, N, 1, tw, lane);
    stockham<5, SIGN>(b, a, N, 8, tw, lane);
    stockham<5, SIGN>(a, b, N, 40, tw, lane);
}
// 100-point line: a -> b
template <int SIGN>
__device__ __forceinline__ void line100(float2 *a, float2 *b, const float2 *tw, int lane) {
    stockham<4, SIGN>(a, b, M, 1, tw, lane);
    stockham<5, SIGN>(b, a, M, 4, tw, lane);
    stockham<5, SIGN>(a, b, M, 20, tw, lane);
}

__device__ __forceinline__ void make_tw200(float2 *tw) {
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        const int r = e < M ? e : e - M;
        const float2 w = make_float2(kTwTable<N>.re[r], kTwTable<N>.im[r]);
        tw[e] = e < M ? w : make_float2(-w.x, -w.y);
    }
}

// every column v <= 100 of buf, inverse (SIGN +) or forward (SIGN -) over u,
// in place; `scale` multiplies the column on the way in
template <int SIGN>
__device__ __forceinline__ void columns(float2 *buf, float2 *sa, float2 *sb, const float2 *tw, int warp, int lane,
                                        float scale = 1.f) {
    for (int k = warp; k < HW; k += NWARP) {
        for (int u = lane; u < N; u += 32) {
            const float2 z = buf[u * HW + k];
            sa[u] = make_float2(z.x * scale, z.y * scale);
        }
        __syncwarp();
        line200<SIGN>(sa, sb, tw, lane);
        for (int u = lane; u < N; u += 32) buf[u * HW + k] = sb[u];
        __syncwarp();
    }
}

// row y of the column-transformed half array back to 200 real values: on
// return sb[n] = (r[2n], r[2n + 1]), n < 100
__device__ __forceinline__ void row_c2r(const float2 *buf, int y, float2 *sa, float2 *sb, const float2 *tw,
                                        int lane) {
    const float2 *row = buf + y * HW;
    for (int k = lane; k < M; k += 32) {
        const float2 c = row[k], cc = c_conj(row[M - k]);
        const float2 e = c_add(c, cc), o = c_mul(c_sub(c, cc), tw[k]);
        sa[k] = make_float2(e.x - o.y, e.y + o.x);   // E + i O
    }
    __syncwarp();
    line100<+1>(sa, sb, tw, lane);
}

__device__ __forceinline__ float hann(int k) { return 0.5f * (1.f - cospif(2.f * k / N)); }

// ---------------------------------------------------------------- pre-processing
__global__ void __launch_bounds__(NT, 1) k_prep_n200(const float *__restrict__ img, PrepArgs a,
                                                     float2 *__restrict__ spec, float *__restrict__ spatial,
                                                     int *__restrict__ degen, const int *__restrict__ active) {
    const int p = blockIdx.x;
    if (active && !active[p]) return;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tw = buf + OFF_TW;
    __shared__ double red[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *sa = buf + OFF_SCR + warp * 2 * N, *sb = sa + N;
    make_tw200(tw);
    const float *src = img + (size_t)p * a.W * a.H;
    float2 *out = spec + (size_t)p * N * HW;
    // statistics: FP32 sums of (x - x0), x0 the crop's first pixel, combined in FP64
    const float x0 = __ldg(src + (size_t)a.oy * a.W + a.ox);
    float s1 = 0.f, s2 = 0.f;
    for (int idx = tid; idx < N * N; idx += NT) {
        const int r = idx / N, c = idx - r * N;
        const float d = __ldg(src + (size_t)(a.oy + r) * a.W + a.ox + c) - x0;
        s1 += d;
        s2 = fmaf(d, d, s2);
    }
    const double m1 = gen::block_sum_f(s1, red) / (N * N), m2 = gen::block_sum_f(s2, red) / (N * N);
    const double mean = x0 + m1, var = m2 - m1 * m1;
    const double sd = var > 0.0 ? sqrt(var) : 0.0;
    bool bad = !(sd > 1e-12 * (1.0 + fabs(mean)));
    double energy = 0.0;
    if (!bad) {
        const float mf = (float)mean, inv = (float)(1.0 / sd);
        // rows: the standardised, windowed row as 100 complex points (x[2n], x[2n + 1]),
        // transformed, then split into its half spectrum X[k] = E[k] + e^{-2 pi i k / 200} O[k]
        for (int y = warp; y < N; y += NWARP) {
            const float *row = src + (size_t)(a.oy + y) * a.W + a.ox;
            const float wy = (a.window ? hann(y) : 1.f) * inv;
            for (int n = lane; n < M; n += 32) {
                const float w0 = a.window ? hann(2 * n) : 1.f, w1 = a.window ? hann(2 * n + 1) : 1.f;
                sa[n] = make_float2((__ldg(row + 2 * n) - mf) * w0 * wy, (__ldg(row + 2 * n + 1) - mf) * w1 * wy);
            }
            __syncwarp();
            line100<-1>(sa, sb, tw, lane);
            for (int k = lane; k <= M; k += 32) {
                const float2 zk = sb[k == M ? 0 : k], zc = c_conj(sb[k == 0 ? 0 : M - k]);
                const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
                const float2 d = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
                const float2 o = make_float2(d.y, -d.x);   // d / i
                buf[y * HW + k] = c_add(e, c_mul(o, tw_at<-1>(tw, k)));
            }
            __syncwarp();
        }
        __syncthreads();
        columns<-1>(buf, sa, sb, tw, warp, lane);
        __syncthreads();
        // band-pass and the filtered energy (columns 1..99 stand for their mirror images too)
        float e = 0.f;
        for (int it = tid; it < N * HW; it += NT) {
            const int u = it / HW, v = it - u * HW;
            const float fu = (float)(u < N / 2 ? u : u - N), fv = (float)(v < N / 2 ? v : v - N);
            const float rho2 = fu * fu + fv * fv;
            const float h = -expm1f(-rho2 * a.inv2shp) * expf(-rho2 * a.inv2slp);
            const float2 X = make_float2(buf[it].x * h, buf[it].y * h);
            buf[it] = X;
            e = fmaf(v == 0 || v == N / 2 ? 1.f : 2.f, X.x * X.x + X.y * X.y, e);
        }
        energy = gen::block_sum_f(e, red);
        bad = !(energy > 0.0);
    }
    if (tid == 0 && degen) degen[p] = bad ? 1 : 0;
    if (bad) {
        for (int idx = tid; idx < N * HW; idx += NT) out[idx] = make_float2(0.f, 0.f);
        if (spatial)
            for (int idx = tid; idx < N * N; idx += NT) spatial[(size_t)p * N * N + idx] = 0.f;
        return;
    }
    const float sc = (float)(1.0 / sqrt(energy));
    for (int it = tid; it < N * HW; it += NT) out[it] = make_float2(buf[it].x * sc, buf[it].y * sc);
    if (!spatial) return;
    // ---- filtered image: the unit-norm spectrum back through the columns and the rows, / N
    columns<+1>(buf, sa, sb, tw, warp, lane, sc);
    __syncthreads();
    const float invn = 1.f / N;
    float2 *sout = reinterpret_cast<float2 *>(spatial + (size_t)p * N * N);
    for (int y = warp; y < N; y += NWARP) {
        row_c2r(buf, y, sa, sb, tw, lane);
        for (int n = lane; n < M; n += 32) sout[y * M + n] = make_float2(sb[n].x * invn, sb[n].y * invn);
        __syncwarp();
    }
}

// ------------------------------------------------------------------- search
// pattern p (blockIdx.y) against the slots [jb, je) (every template, or the
// pattern's candidate list); one template per pass; the best into keys[p]
__global__ void __launch_bounds__(NT, 1) k_search_n200(const float2 *__restrict__ St, int T,
                                                       const float2 *__restrict__ Sp, const int *__restrict__ degen,
                                                       int per_cta, unsigned long long *__restrict__ keys,
                                                       float *__restrict__ peaks_all, const int *__restrict__ cand,
                                                       int kc) {
    const int p = blockIdx.y;
    if (degen[p]) return;
    const int n = cand ? kc : T;
    const int jb = blockIdx.x * per_cta, je = min(n, jb + per_cta);
    if (jb >= je) return;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tw = buf + OFF_TW;
    __shared__ float rmax[NWARP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *sa = buf + OFF_SCR + warp * 2 * N, *sb = sa + N;
    make_tw200(tw);
    const float2 *sp = Sp + (size_t)p * N * HW;
    float best_v = -INFINITY;
    int best_t = -1;
    for (int j = jb; j < je; ++j) {
        const int t = cand ? cand[(size_t)p * kc + j] : j;
        if (t < 0) {   // an empty candidate slot (uniform over the CTA)
            if (peaks_all && tid == 0) peaks_all[(size_t)p * n + j] = -INFINITY;
            continue;
        }
        const float2 *st = St + (size_t)t * N * HW;
        __syncthreads();   // the previous template's rows are read; the twiddles are in place
        for (int it = tid; it < N * HW; it += NT) buf[it] = c_mulcj(__ldg(st + it), __ldg(sp + it));
        __syncthreads();
        columns<+1>(buf, sa, sb, tw, warp, lane);
        __syncthreads();
        float m = -INFINITY;
        for (int y = warp; y < N; y += NWARP) {
            row_c2r(buf, y, sa, sb, tw, lane);
            for (int k = lane; k < M; k += 32) m = fmaxf(m, fmaxf(sb[k].x, sb[k].y));
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) rmax[warp] = m;
        __syncthreads();
        if (tid == 0) {
            float v = rmax[0];
            for (int w = 1; w < NWARP; ++w) v = fmaxf(v, rmax[w]);
            if (peaks_all) peaks_all[(size_t)p * n + j] = v;
            if (v > best_v || (v == best_v && t < best_t)) {
                best_v = v;
                best_t = t;
            }
        }
    }
    if (tid == 0 && best_t >= 0) atomicMax(keys + p, pack_key(best_v, best_t));
}

__device__ __forceinline__ float parabola200(float cm, float c0, float cp) {
    const float den = cm - 2.f * c0 + cp;
    if (!(den < 0.f)) return 0.f;
    const float d = (cm - cp) / (2.f * den);
    return fminf(0.5f, fmaxf(-0.5f, d));
}

// ------------------------------------------------------- single-surface peak
// integer argmax of pattern p's surface against template tidx[p] (ties ->
// lowest row-major index), the peak value and the 3-point parabola per axis;
// the three rows around the argmax are recomputed from the column-transformed
// half array for the neighbours
__global__ void __launch_bounds__(NT, 1) k_pair_peak_n200(const float2 *__restrict__ St,
                                                          const int *__restrict__ tidx,
                                                          const float2 *__restrict__ Sp,
                                                          const int *__restrict__ degen,
                                                          const int *__restrict__ active, int P,
                                                          float *__restrict__ peak, float *__restrict__ shift,
                                                          int *__restrict__ argmax) {
    const int p = blockIdx.x;
    if (p >= P || (active && !active[p])) return;
    const int t = tidx ? tidx[p] : p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if ((degen && degen[p]) || t < 0) {
        if (tid == 0) {
            peak[p] = 0.f;
            shift[2 * p] = 0.f;
            shift[2 * p + 1] = 0.f;
        }
        return;
    }
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tw = buf + OFF_TW;
    __shared__ float rv[NWARP];
    __shared__ int ri[NWARP];
    __shared__ int s_best;
    float2 *sa = buf + OFF_SCR + warp * 2 * N, *sb = sa + N;
    make_tw200(tw);
    const float2 *st = St + (size_t)t * N * HW, *sp = Sp + (size_t)p * N * HW;
    for (int it = tid; it < N * HW; it += NT) buf[it] = c_mulcj(__ldg(st + it), __ldg(sp + it));
    __syncthreads();
    columns<+1>(buf, sa, sb, tw, warp, lane);
    __syncthreads();
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int y = warp; y < N; y += NWARP) {
        row_c2r(buf, y, sa, sb, tw, lane);
        for (int k = lane; k < M; k += 32) {
            const float2 z = sb[k];
            const int i0 = y * N + 2 * k;
            if (z.x > bv || (z.x == bv && i0 < bi)) { bv = z.x; bi = i0; }
            if (z.y > bv || (z.y == bv && i0 + 1 < bi)) { bv = z.y; bi = i0 + 1; }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        float b = rv[0];
        int i0 = ri[0];
        for (int w = 1; w < NWARP; ++w)
            if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
        s_best = i0;
    }
    __syncthreads();
    if (warp != 0) return;
    const int i0 = s_best, y0 = i0 / N, x0 = i0 - y0 * N;
    // the surface at row y, column x from a row just transformed into sb
    auto at = [&](int x) {
        const float2 z = sb[x >> 1];
        return (x & 1) ? z.y : z.x;
    };
    row_c2r(buf, (y0 + N - 1) % N, sa, sb, tw, lane);
    const float cym = at(x0);
    __syncwarp();
    row_c2r(buf, (y0 + 1) % N, sa, sb, tw, lane);
    const float cyp = at(x0);
    __syncwarp();
    row_c2r(buf, y0, sa, sb, tw, lane);
    const float c0 = at(x0), cxm = at((x0 + N - 1) % N), cxp = at((x0 + 1) % N);
    if (lane == 0) {
        peak[p] = c0;
        shift[2 * p] = (float)(x0 < N / 2 ? x0 : x0 - N) + parabola200(cxm, c0, cxp);
        shift[2 * p + 1] = (float)(y0 < N / 2 ? y0 : y0 - N) + parabola200(cym, c0, cyp);
        if (argmax) argmax[p] = i0;
    }
}

template <typename K>
cudaError_t smem_attr(K kern) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
}

}  // namespace

cudaError_t launch_prep_n200(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                             const int *active, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (a.N != N) return cudaErrorInvalidValue;
    cudaError_t e = smem_attr(k_prep_n200);
    if (e != cudaSuccess) return e;
    k_prep_n200<<<P, NT, SMEM_BYTES, st>>>(img, a, spec, spatial, degen, active);
    return cudaGetLastError();
}

cudaError_t launch_search_n200(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                               unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st,
                               const int *cand, int kc) {
    const int n = cand ? kc : T;
    if (P <= 0 || n <= 0) return cudaSuccess;
    cudaError_t e = smem_attr(k_search_n200);
    if (e != cudaSuccess) return e;
    // enough CTAs to fill the GPU twice over, at least 4 templates each
    const long want = (long)num_sms * 2;
    int chunks = (int)((want + P - 1) / P);
    chunks = max(1, min(chunks, (n + 3) / 4));
    int per = (n + chunks - 1) / chunks;
    chunks = (n + per - 1) / per;
    dim3 grid(chunks, P);
    k_search_n200<<<grid, NT, SMEM_BYTES, st>>>(St, T, Sp, degen, per, keys, peaks_all, cand, kc);
    return cudaGetLastError();
}

cudaError_t launch_pair_peak_n200(const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                  const int *active, int P, float *peak, float *shift, int *argmax, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    cudaError_t e = smem_attr(k_pair_peak_n200);
    if (e != cudaSuccess) return e;
    k_pair_peak_n200<<<P, NT, SMEM_BYTES, st>>>(St, tidx, Sp, degen, active, P, peak, shift, argmax);
    return cudaGetLastError();
}
