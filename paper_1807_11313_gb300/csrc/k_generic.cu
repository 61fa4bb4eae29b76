// Pre-processing, the all-sides search kernel and the single-surface peak
// kernel for N in {16, 32, 64, 96, 128, 160}.  The search and peak kernels
// hold one N x N complex array in shared memory (rows padded to N + 1) and
// transform its lines with the warp line FFT (registers and shuffles for
// N = R x 32 >= 64, mixed radix at 96 and 160; radix-2 butterflies spread
// over the lanes below 64); the pre-processing transforms two real images per
// complex transform (rows paired for 2^k sides, whole images for 96 and 160).
//
// Paper: FFT section (Eq. 4 transform, filtering, windowing, normalisation by
// the autocorrelations), Eqs. 3 and 6 (correlation surface), peak up-sampling.
#include "common.cuh"
#include "generic.cuh"
#include "kernels.cuh"
#include "oct64.cuh"
#include "project.cuh"

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
template <int N>
__host__ __device__ constexpr int search_threads() { return N >= 128 ? 1024 : kThreads; }

// PROJ: the image is projected from the master pattern (ps) while it is
// loaded, instead of read from img
template <int N, int PT = prep_threads<N>(), bool PROJ = false>
__global__ void __launch_bounds__(PT) k_prep_real(const float *__restrict__ img, PrepArgs a,
                                                        float2 *__restrict__ spec, float *__restrict__ spatial,
                                                        int *__restrict__ degen, const int *__restrict__ active,
                                                        ProjSrc ps) {
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
    // per-index tables: the Hann window, and the band-pass as a product of
    // per-frequency factors (e(f) = expm1(-f^2 / 2 s_h^2), b(f) = exp(-f^2 / 2 s_l^2):
    // 1 - exp(-(x_u + x_v)) = -(e_u + e_v + e_u e_v), free of cancellation near DC)
    __shared__ float win[N], fe[N / 2 + 1], fb[N / 2 + 1];
    const int p = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < N; i += PT) win[i] = a.window ? 0.5f * (1.f - cospif(2.f * i / N)) : 1.f;
    for (int i = tid; i <= N / 2; i += PT) {
        const float f2 = (float)(i * i);
        fe[i] = expm1f(-f2 * a.inv2shp);
        fb[i] = expf(-f2 * a.inv2slp);
    }
    const float *src = img + (size_t)p * a.W * a.H;
    float2 *out = spec + (size_t)p * N * HW;
    make_twiddles<N>(twN, -1);
    make_twiddles<N>(twNi, +1);
    make_twiddles<H>(twH, -1);
    make_twiddles<H>(twHi, +1);
    // ---- load (rows 2pr, 2pr+1 into the real and imaginary parts of buf row pr) and statistics:
    // one pass of FP32 sums of (x - x0), x0 the crop's first pixel (a constant crop has exactly
    // zero variance; the shift keeps the per-thread sums well conditioned), combined in FP64
    __shared__ proj::Frame fr;
    proj::Frame f{};   // in registers: the loops below store to shared memory, which could alias fr
    if constexpr (PROJ) {
        if (tid == 0) proj::frame(ps.quats + 4 * (size_t)p, ps.pcs ? ps.pcs + 3 * (size_t)p : nullptr, ps.a, fr);
        __syncthreads();
        f = fr;
    }
    auto pixel = [&](int r, int c) -> float {   // image pixel (a.oy + r, a.ox + c)
        if constexpr (PROJ)
            return proj::pixel(f, ps.master, ps.M, ps.a, a.oy + r, a.ox + c);
        else
            return src[(size_t)(a.oy + r) * a.W + a.ox + c];
    };
    const float x0 = pixel(0, 0);
    float s1 = 0.f, s2 = 0.f;
    auto take = [&](int r, int c, float v) {
        reinterpret_cast<float *>(buf + (r >> 1) * LD + c)[r & 1] = v;
        const float d = v - x0;
        s1 += d;
        s2 = fmaf(d, d, s2);
    };
    if constexpr (PROJ && PT % N == 0) {
        // every pixel of this thread lies in column tid mod N: its column part once
        const int c = tid % N;
        const proj::Col col = proj::column(f, ps.a, a.ox + c);
        for (int r = tid / N; r < N; r += PT / N) take(r, c, proj::pixel(f, col, ps.master, ps.M, ps.a, a.oy + r));
    } else {
        for (int idx = tid; idx < N * N; idx += PT) {
            const int r = idx / N, c = idx % N;
            take(r, c, pixel(r, c));
        }
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
            const float wc = win[c] * inv, w0 = win[2 * pr], w1 = win[2 * pr + 1];
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
            const int iu = u <= N / 2 ? u : N - u;   // |f_u|; |f_v| = v (v <= N/2)
            const float eu = fe[iu], ev = fe[v];
            const float h = -(eu + ev + eu * ev) * (fb[iu] * fb[v]);
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

// --------------------------------------------------------------------------
// pre-processing of two images per CTA for the native 96 x 96 and 160 x 160
// sides: image A in the real and image B in the imaginary part of one complex
// N x N array in shared memory (rows padded to N + 1), one complex 2-D
// transform (mixed-radix register line FFTs), then the two spectra split by
// Hermitian symmetry, X_A = (Z(k) + conj Z(-k)) / 2, X_B = (Z(k) - conj
// Z(-k)) / 2i.  In place, X_A(u, v) stays at (u, v) and X_B(u, v) moves to the
// mirror (-u, -v) for 0 < v < N/2 (one thread owns both cells); columns 0 and
// N/2 (their mirrors lie in the same column) go to four separate columns.  The
// spatial outputs come back together from Z' = X_A' + i X_B'.
// --------------------------------------------------------------------------
constexpr int kPrepCplxThreads = 512;
template <int N>
constexpr size_t smem_prep_cplx() {
    return sizeof(float2) * ((size_t)N * (N + 1) + N + 4 * N);
}

template <int N>
__global__ void __launch_bounds__(kPrepCplxThreads, 1) k_prep_cplx(const float *__restrict__ img, int P, PrepArgs a,
                                                                float2 *__restrict__ spec,
                                                                float *__restrict__ spatial,
                                                                int *__restrict__ degen,
                                                                const int *__restrict__ active) {
    constexpr int LD = N + 1, HW = N / 2 + 1, NT = kPrepCplxThreads, H2 = N / 2;
    extern __shared__ float4 smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *twf = buf + N * LD, *twi = twf + N / 2;
    float2 *cA0 = twi + N / 2, *cAH = cA0 + N, *cB0 = cAH + N, *cBH = cB0 + N;
    __shared__ double red[33];
    const int tid = threadIdx.x;
    const int pa = 2 * blockIdx.x, pb = pa + 1;
    const bool ha = pa < P && (!active || active[pa]);
    const bool hb = pb < P && (!active || active[pb]);
    if (!ha && !hb) return;   // uniform over the CTA
    make_twiddles<N>(twf, -1);
    make_twiddles<N>(twi, +1);
    const size_t isz = (size_t)a.W * a.H, off = (size_t)a.oy * a.W + a.ox;
    const float *sa = img + (size_t)(ha ? pa : pb) * isz + off, *sb = img + (size_t)(hb ? pb : pa) * isz + off;
    // ---- load both crops; FP32 statistics of (x - x0), x0 each crop's first pixel
    const float xa0 = ha ? __ldg(sa) : 0.f, xb0 = hb ? __ldg(sb) : 0.f;
    float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
    for (int idx = tid; idx < N * N; idx += NT) {
        const int r = idx / N, c = idx - r * N;
        const float va = ha ? __ldg(sa + (size_t)r * a.W + c) : 0.f;
        const float vb = hb ? __ldg(sb + (size_t)r * a.W + c) : 0.f;
        buf[r * LD + c] = make_float2(va, vb);
        const float da = va - xa0, db = vb - xb0;
        a1 += da;
        a2 = fmaf(da, da, a2);
        b1 += db;
        b2 = fmaf(db, db, b2);
    }
    const double A1 = block_sum_f(a1, red) / (N * N), A2 = block_sum_f(a2, red) / (N * N);
    const double B1 = block_sum_f(b1, red) / (N * N), B2 = block_sum_f(b2, red) / (N * N);
    const double meanA = xa0 + A1, varA = A2 - A1 * A1, sdA = varA > 0.0 ? sqrt(varA) : 0.0;
    const double meanB = xb0 + B1, varB = B2 - B1 * B1, sdB = varB > 0.0 ? sqrt(varB) : 0.0;
    bool badA = !ha || !(sdA > 1e-12 * (1.0 + fabs(meanA)));
    bool badB = !hb || !(sdB > 1e-12 * (1.0 + fabs(meanB)));
    // ---- standardise and window (a degenerate crop becomes zeros)
    {
        const float mA = (float)meanA, iA = badA ? 0.f : (float)(1.0 / sdA);
        const float mB = (float)meanB, iB = badB ? 0.f : (float)(1.0 / sdB);
        for (int idx = tid; idx < N * N; idx += NT) {
            const int r = idx / N, c = idx - r * N;
            const float w = a.window ? 0.25f * (1.f - cospif(2.f * r / N)) * (1.f - cospif(2.f * c / N)) : 1.f;
            const float2 z = buf[r * LD + c];
            buf[r * LD + c] = make_float2((z.x - mA) * iA * w, (z.y - mB) * iB * w);
        }
    }
    __syncthreads();
    smem_fft_lines<N>(buf, N, LD, 1, twf);   // rows
    __syncthreads();
    smem_fft_lines<N>(buf, N, 1, LD, twf);   // columns
    __syncthreads();
    auto filt = [&](int u, int v) {
        const float fu = (float)(u < N / 2 ? u : u - N), fv = (float)(v < N / 2 ? v : v - N);
        const float rho2 = fu * fu + fv * fv;
        return -expm1f(-rho2 * a.inv2shp) * expf(-rho2 * a.inv2slp);
    };
    // ---- split, filter, energies (bins 1..N/2-1 stand for their mirrors too)
    float eA = 0.f, eB = 0.f;
    for (int it = tid; it < N * (H2 - 1); it += NT) {
        const int u = it / (H2 - 1), v = 1 + it % (H2 - 1), um = (N - u) % N, vm = N - v;
        const float2 z = buf[u * LD + v], zm = buf[um * LD + vm];
        const float h = filt(u, v);
        const float2 XA = make_float2(0.5f * h * (z.x + zm.x), 0.5f * h * (z.y - zm.y));
        const float2 XB = make_float2(0.5f * h * (z.y + zm.y), 0.5f * h * (zm.x - z.x));
        eA = fmaf(2.f, XA.x * XA.x + XA.y * XA.y, eA);
        eB = fmaf(2.f, XB.x * XB.x + XB.y * XB.y, eB);
        buf[u * LD + v] = XA;
        buf[um * LD + vm] = XB;
    }
    for (int it = tid; it < 2 * N; it += NT) {   // columns 0 and N/2 (not touched by the loop above)
        const int u = it % N, v = it < N ? 0 : H2, um = (N - u) % N;
        const float2 z = buf[u * LD + v], zm = buf[um * LD + v];
        const float h = filt(u, v);
        const float2 XA = make_float2(0.5f * h * (z.x + zm.x), 0.5f * h * (z.y - zm.y));
        const float2 XB = make_float2(0.5f * h * (z.y + zm.y), 0.5f * h * (zm.x - z.x));
        eA += XA.x * XA.x + XA.y * XA.y;
        eB += XB.x * XB.x + XB.y * XB.y;
        (v ? cAH : cA0)[u] = XA;
        (v ? cBH : cB0)[u] = XB;
    }
    const double EA = block_sum_f(eA, red), EB = block_sum_f(eB, red);   // its barriers order the writes above
    badA = badA || !(EA > 0.0);
    badB = badB || !(EB > 0.0);
    if (tid == 0 && degen) {
        if (ha) degen[pa] = badA ? 1 : 0;
        if (hb) degen[pb] = badB ? 1 : 0;
    }
    const float sA = badA ? 0.f : (float)(1.0 / sqrt(EA)), sB = badB ? 0.f : (float)(1.0 / sqrt(EB));
    float2 *oa = spec + (size_t)pa * N * HW, *ob = spec + (size_t)pb * N * HW;
    for (int it = tid; it < N * HW; it += NT) {
        const int u = it / HW, v = it - u * HW;
        float2 XA, XB;
        if (v == 0) { XA = cA0[u]; XB = cB0[u]; }
        else if (v == H2) { XA = cAH[u]; XB = cBH[u]; }
        else { XA = buf[u * LD + v]; XB = buf[((N - u) % N) * LD + N - v]; }
        if (ha) oa[it] = make_float2(XA.x * sA, XA.y * sA);
        if (hb) ob[it] = make_float2(XB.x * sB, XB.y * sB);
    }
    if (!spatial) return;
    __syncthreads();
    // ---- spatial images: Z' = sA X_A + i sB X_B over the full spectrum, one inverse transform
    for (int it = tid; it < N * (H2 - 1); it += NT) {
        const int u = it / (H2 - 1), v = 1 + it % (H2 - 1), um = (N - u) % N, vm = N - v;
        const float2 XA = buf[u * LD + v], XB = buf[um * LD + vm];
        // Z'(u, v) = sA XA + i sB XB; Z'(-u, -v) = sA conj XA + i sB conj XB
        buf[u * LD + v] = make_float2(sA * XA.x - sB * XB.y, sA * XA.y + sB * XB.x);
        buf[um * LD + vm] = make_float2(sA * XA.x + sB * XB.y, -sA * XA.y + sB * XB.x);
    }
    for (int it = tid; it < 2 * N; it += NT) {
        const int u = it % N, v = it < N ? 0 : H2;
        const float2 XA = (v ? cAH : cA0)[u], XB = (v ? cBH : cB0)[u];
        buf[u * LD + v] = make_float2(sA * XA.x - sB * XB.y, sA * XA.y + sB * XB.x);
    }
    __syncthreads();
    smem_fft_lines<N>(buf, N, LD, 1, twi);   // rows back
    __syncthreads();
    smem_fft_lines<N>(buf, N, 1, LD, twi);   // columns back
    __syncthreads();
    const float invn = 1.f / N;
    for (int idx = tid; idx < N * N; idx += NT) {
        const int r = idx / N, c = idx - r * N;
        const float2 z = buf[r * LD + c];
        if (ha) spatial[(size_t)pa * N * N + idx] = z.x * invn;
        if (hb) spatial[(size_t)pb * N * N + idx] = z.y * invn;
    }
}

template <int N>
__global__ void __launch_bounds__(search_threads<N>()) k_search_generic(const float2 *__restrict__ St, int T,
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
    search_body<N, (search_threads<N>() <= 512)>(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc);
}

// N = 64: the eight-lane-group body (8 x 8 line transforms) on 128-thread
// CTAs, several resident per SM
constexpr int kOctThreads = 128;
__global__ void __launch_bounds__(kOctThreads) k_search_oct64(const float2 *__restrict__ St, int T,
                                                             const float2 *__restrict__ Sp,
                                                             const int *__restrict__ degen, int pairs_per_cta,
                                                             unsigned long long *__restrict__ keys,
                                                             float *__restrict__ peaks_all,
                                                             const int *__restrict__ cand, int kc) {
    const int p = blockIdx.y;
    if (degen[p]) return;
    const int npairs = ((cand ? kc : T) + 1) / 2;
    const int pb = blockIdx.x * pairs_per_cta, pe = min(npairs, pb + pairs_per_cta);
    o64::search_body(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc, gen::cta_group());
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
    // each stored value (u, v <= N/2) gives Z(u, v) = X1 + i X2 and, for 0 < v < N/2,
    // Z(-u, -v) = conj X1 + i conj X2 (Hermitian symmetry of both surfaces)
    for (int k = tid; k < N * HW; k += QT) {
        const int u = k / HW, v = k - u * HW;
        float2 x1 = c_mulcj(ta[k], qa[k]), x2 = c_mulcj(tb[k], qb[k]);
        x1 = make_float2(x1.x * fa, x1.y * fa);
        x2 = make_float2(x2.x * fb, x2.y * fb);
        buf[u * LD + v] = make_float2(x1.x - x2.y, x1.y + x2.x);
        if (v > 0 && v < N / 2) buf[(u == 0 ? 0 : N - u) * LD + (N - v)] = make_float2(x1.x + x2.y, -x1.y + x2.x);
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
        const float cxm = at(y0, (x0 + N - 1) % N), cxp = at(y0, (x0 + 1) % N);
        const float cym = at((y0 + N - 1) % N, x0), cyp = at((y0 + 1) % N, x0);
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
    k_prep_real<N><<<P, prep_threads<N>(), sm, st>>>(img, a, spec, spatial, degen, active, ProjSrc{});
    return cudaGetLastError();
}

template <int N>
cudaError_t prep_projected_n(const ProjSrc &src, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                             const int *active, cudaStream_t st) {
    const size_t sm = smem_prep_real<N>();
    auto *k = k_prep_real<N, prep_threads<N>(), true>;
    cudaError_t e = set_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<P, prep_threads<N>(), sm, st>>>(nullptr, a, spec, spatial, degen, active, src);
    return cudaGetLastError();
}

template <int N>
cudaError_t prep_cplx_n(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                        const int *active, cudaStream_t st) {
    const size_t sm = smem_prep_cplx<N>();
    cudaError_t e = set_smem(k_prep_cplx<N>, sm);
    if (e != cudaSuccess) return e;
    k_prep_cplx<N><<<(P + 1) / 2, kPrepCplxThreads, sm, st>>>(img, P, a, spec, spatial, degen, active);
    return cudaGetLastError();
}

template <int N>
cudaError_t search_n(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                     unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st,
                     const int *cand = nullptr, int kc = 0) {
    const int npairs = ((cand ? kc : T) + 1) / 2;
    if constexpr (N == 64) {   // 128-thread CTAs: enough to fill every SM four deep a few times over
        const size_t sm = o64::smem_bytes(kOctThreads);
        cudaError_t e = set_smem(k_search_oct64, sm);
        if (e != cudaSuccess) return e;
        const long want = (long)num_sms * 32;
        int chunks = (int)((want + P - 1) / P);
        chunks = max(1, min(chunks, (npairs + 3) / 4));
        int ppc = (npairs + chunks - 1) / chunks;
        chunks = (npairs + ppc - 1) / ppc;
        k_search_oct64<<<dim3(chunks, P), kOctThreads, sm, st>>>(St, T, Sp, degen, ppc, keys, peaks_all, cand, kc);
        return cudaGetLastError();
    }
    size_t sm = gen::smem_bytes<N>();
    cudaError_t e = set_smem(k_search_generic<N>, sm);
    if (e != cudaSuccess) return e;
    // enough CTAs to fill the GPU a few times over, at least 4 pairs each
    long want = (long)num_sms * 8;
    int chunks = (int)((want + P - 1) / P);
    chunks = max(1, min(chunks, (npairs + 3) / 4));
    int ppc = (npairs + chunks - 1) / chunks;
    chunks = (npairs + ppc - 1) / ppc;
    dim3 grid(chunks, P);
    k_search_generic<N><<<grid, search_threads<N>(), sm, st>>>(St, T, Sp, degen, ppc, keys, peaks_all, cand, kc);
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
        case 96: return prep_cplx_n<96>(img, P, a, spec, spatial, degen, active, st);
        case 160: return prep_cplx_n<160>(img, P, a, spec, spatial, degen, active, st);
        case 200: return launch_prep_n200(img, P, a, spec, spatial, degen, active, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prep_projected(const ProjSrc &src, int P, const PrepArgs &a, float2 *spec, float *spatial,
                                  int *degen, const int *active, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (src.a.nx != a.W || src.a.ny != a.H) return cudaErrorInvalidValue;
    ProjSrc s = src;   // the rotation's cosine and sine once, on the host (as launch_project)
    s.a.ca = cos(src.a.alpha);
    s.a.sa = sin(src.a.alpha);
    switch (a.N) {
        case 16: return prep_projected_n<16>(s, P, a, spec, spatial, degen, active, st);
        case 32: return prep_projected_n<32>(s, P, a, spec, spatial, degen, active, st);
        case 64: return prep_projected_n<64>(s, P, a, spec, spatial, degen, active, st);
        case 128: return prep_projected_n<128>(s, P, a, spec, spatial, degen, active, st);
        default: return cudaErrorNotSupported;
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
        case 96: return search_n<96>(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
        case 160: return search_n<160>(St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
        case 200: return launch_search_n200(St, T, Sp, degen, P, keys, peaks_all, num_sms, st, nullptr, 0);
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
        case 96: return search_n<96>(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
        case 160: return search_n<160>(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
        case 200: return launch_search_n200(St, 0, Sp, degen, P, keys, peaks, num_sms, st, cand, kc);
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
        case 96: return pair_peak_n<96>(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        case 160: return pair_peak_n<160>(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        case 200: return launch_pair_peak_n200(St, tidx, Sp, degen, active, P, peak, shift, argmax, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_keys_to_best(const unsigned long long *keys, int P, int *best, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_keys_to_best<<<(P + 255) / 256, 256, 0, st>>>(keys, P, best);
    return cudaGetLastError();
}
