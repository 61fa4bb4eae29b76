// Geometry and refinement kernels: gnomonic reprojection of the master
// pattern, log-polar resampling, the angular correlation, float64 orientation
// updates and the cubic disorientation.
//
// Paper: "SO(3) Library Generation" (reprojection of the master pattern),
// "Orientation and Pattern Centre Refinement" (Eq. 7, Fig. 6: shifts to
// rotations about detector x / y, log-polar transform for z), second
// "Equation 6" (disorientation with the 24 cubic operators).
#include "common.cuh"
#include "line_fft.cuh"
#include "kernels.cuh"
#include "project.cuh"

namespace {

// ----------------------------------------------------------- quaternions
struct Q { double w, x, y, z; };

__device__ __forceinline__ Q qmul(const Q &a, const Q &b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
            a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
            a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ Q qconj(const Q &a) { return {a.w, -a.x, -a.y, -a.z}; }
__device__ __forceinline__ Q qcanon(Q a) {
    double s = sqrt(a.w * a.w + a.x * a.x + a.y * a.y + a.z * a.z);
    if (a.w < 0) s = -s;
    return {a.w / s, a.x / s, a.y / s, a.z / s};
}
__device__ __forceinline__ Q qload(const double *p) { return {p[0], p[1], p[2], p[3]}; }
__device__ __forceinline__ void qstore(double *p, const Q &a) {
    p[0] = a.w; p[1] = a.x; p[2] = a.y; p[3] = a.z;
}
// orientation whose template is the template of q rotated by the
// detector-frame rotation R: q (x) qs (x) conj(R) (x) conj(qs), qs = detector
// -> sample rotation about x by alpha
__device__ __forceinline__ Q rotate_in_detector(const Q &q, const Q &R, double alpha) {
    double s, c;
    sincos(0.5 * alpha, &s, &c);
    const Q qs = {c, s, 0.0, 0.0};
    return qcanon(qmul(qmul(qmul(q, qs), qconj(R)), qconj(qs)));
}

// ---------------------------------------------------------- projection
__global__ void __launch_bounds__(256) k_project(const float *__restrict__ master, int M,
                                                 const double *__restrict__ quats,
                                                 const double *__restrict__ pcs,
                                                 const int *__restrict__ active, ProjArgs a,
                                                 float *__restrict__ out) {
    const int p = blockIdx.y;
    if (active && !active[p]) return;
    __shared__ proj::Frame fr;
    if (threadIdx.x == 0) proj::frame(quats + 4 * (size_t)p, pcs ? pcs + 3 * (size_t)p : nullptr, a, fr);
    __syncthreads();
    const proj::Frame f = fr;   // in registers: the loop's stores could alias shared memory
    const int npx = a.nx * a.ny;
    float *dst = out + (size_t)p * npx;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < npx; idx += gridDim.x * blockDim.x) {
        const int i = idx / a.nx, j = idx % a.nx;
        dst[idx] = proj::pixel(f, master, M, a, i, j);
    }
}

// ------------------------------------------------------------ log-polar
// sample idx = m neta + l sits at radius rmin (rmax / rmin)^(m / (nr - 1)) and
// angle 2 pi l / neta about the image centre; o = y0 N + x0 is its bilinear
// corner and (tx, ty) its weights (lr = log(rmax / rmin))
struct LpPos {
    int o;
    float tx, ty;
};
__device__ __forceinline__ LpPos lp_pos(int idx, int N, int nr, int neta, float rmin, float lr) {
    const float c = 0.5f * N - 0.5f;
    const int m = idx / neta, l = idx % neta;
    const float r = rmin * expf(lr * (nr > 1 ? (float)m / (nr - 1) : 0.f));
    float sn, cs;
    sincospif(2.f * l / neta, &sn, &cs);
    const float fx = c + r * cs, fy = c - r * sn;
    int x0 = (int)floorf(fx), y0 = (int)floorf(fy);
    x0 = min(max(x0, 0), N - 2);
    y0 = min(max(y0, 0), N - 2);
    return LpPos{y0 * N + x0, fx - x0, fy - y0};
}
__device__ __forceinline__ float lp_bilinear(const float *g, int N, const LpPos &q) {
    return (1.f - q.ty) * ((1.f - q.tx) * g[0] + q.tx * g[1]) + q.ty * ((1.f - q.tx) * g[N] + q.tx * g[N + 1]);
}

// sides above the shared-memory limit: each thread samples one position of
// kLpPats images (the position, one expf and one sincospif, computed once for
// all of them) straight from global memory
constexpr int kLpPats = 8;
__global__ void __launch_bounds__(256) k_logpolar(const float *__restrict__ spatial,
                                                  const int *__restrict__ active, int P, int N, int nr,
                                                  int neta, float rmin, float rmax, float *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nr * neta) return;
    const LpPos q = lp_pos(idx, N, nr, neta, rmin, logf(rmax / rmin));
    const int p1 = min(P, (int)(blockIdx.y + 1) * kLpPats);
    for (int p = blockIdx.y * kLpPats; p < p1; ++p) {
        if (active && !active[p]) continue;
        out[(size_t)p * nr * neta + idx] = lp_bilinear(spatial + (size_t)p * N * N + q.o, N, q);
    }
}

// sides up to kLpSmemSide: one image per CTA, read from HBM once with
// coalesced 16-byte loads into shared memory and sampled there (the samples'
// scattered bilinear reads then cost shared-memory wavefronts, not sectors)
constexpr int kLpSmemSide = 160;
__global__ void __launch_bounds__(256) k_logpolar_img(const float *__restrict__ spatial,
                                                      const int *__restrict__ active, int N, int nr, int neta,
                                                      float rmin, float rmax, float *__restrict__ out) {
    extern __shared__ float4 lp_img4[];
    const int p = blockIdx.x;
    if (active && !active[p]) return;
    const float4 *src = reinterpret_cast<const float4 *>(spatial + (size_t)p * N * N);
    for (int i = threadIdx.x; i < N * N / 4; i += blockDim.x) lp_img4[i] = src[i];
    __syncthreads();
    const float *img = reinterpret_cast<const float *>(lp_img4);
    const float lr = logf(rmax / rmin);
    float *dst = out + (size_t)p * nr * neta;
    for (int idx = threadIdx.x; idx < nr * neta; idx += blockDim.x) {
        const LpPos q = lp_pos(idx, N, nr, neta, rmin, lr);
        dst[idx] = lp_bilinear(img + q.o, N, q);
    }
}

// FP32 partial per thread: warp sums in FP32, the warps' sums in FP64
__device__ double block_sum_fd(float v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += sh[k];
        sh[32] = s;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float parabola(float cm, float c0, float cp) {
    float den = cm - 2.f * c0 + cp;
    if (!(den < 0.f)) return 0.f;
    float d = (cm - cp) / (2.f * den);
    return fminf(0.5f, fmaxf(-0.5f, d));
}

// ------------------------------------------------ angular correlation + Z
// c(D) = sum_m sum_l a[m][l] b[m][(l + D) mod neta] / (|a| |b|) on mean-free
// log-polar images (a = template, b = pattern), by the correlation theorem:
// each warp transforms radii m = warp, warp + 8, ... as one complex line
// z = a_m + i b_m, splits A_m and B_m by Hermitian symmetry and accumulates
// C[k] = sum_m conj(A_m[k]) B_m[k] (k <= neta/2) in registers; the warps'
// eight sums are added and one inverse transform of the Hermitian C
// gives c(D) for every shift.  neta log neta work per radius instead of neta^2.
constexpr int kEtaThreads = 256, kEtaWarps = kEtaThreads / 32, kMaxLpWindows = 16;

template <int NETA>
__global__ void __launch_bounds__(kEtaThreads, NETA >= 512 ? 2 : 3) k_eta_update(const float *__restrict__ lpT,
                                                            const float *__restrict__ lpP, int nr, int windows,
                                                            const double *__restrict__ q0s,
                                                            const double *__restrict__ q1s,
                                                            double alpha, double tol_deg,
                                                            int *__restrict__ active,
                                                            int *__restrict__ iters,
                                                            double *__restrict__ q_out) {
    constexpr int H = NETA / 2 + 1, KPL = (H + 31) / 32;   // spectrum bins, bins per lane
    const int p = blockIdx.x;
    if (!active[p]) return;
    __shared__ float2 line[kEtaWarps][NETA];   // per-warp lines, then per-warp sums C (k < H)
    __shared__ float2 tw[NETA / 2], twi[NETA / 2];
    __shared__ float2 zc[NETA];
    __shared__ float cfin[NETA];
    __shared__ double red[33];
    __shared__ double wshift[kMaxLpWindows];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float *ga = lpT + (size_t)p * nr * NETA, *gb = lpP + (size_t)p * nr * NETA;
    linefft::make_tw<NETA>(tw, -1);
    linefft::make_tw<NETA>(twi, +1);
    __syncthreads();   // the twiddle tables
    constexpr bool kRegLine = NETA >= 64;   // register warp transforms (NETA = R x 32)
    WarpFftTw<kRegLine ? NETA : 64> wf;
    if constexpr (kRegLine) wf.load(tw, lane);
    float2 *z = line[w];
    // radial window b holds radii [b nr / W, (b + 1) nr / W); each is correlated along eta on its own
    for (int b = 0; b < windows; ++b) {
        const int m0 = b * nr / windows, m1 = (b + 1) * nr / windows;
        const int i0 = m0 * NETA, i1 = m1 * NETA;
        float s1 = 0.f, s2 = 0.f;
        for (int i = i0 + tid; i < i1; i += kEtaThreads) { s1 += ga[i]; s2 += gb[i]; }
        const float ma = (float)(block_sum_fd(s1, red) / (i1 - i0));
        const float mb = (float)(block_sum_fd(s2, red) / (i1 - i0));
        float2 acc[KPL];
#pragma unroll
        for (int j = 0; j < KPL; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int m = m0 + w; m < m1; m += kEtaWarps) {
            // forward: Z[k] = sum_l z[l] e^{-2 pi i k l / NETA}
            if constexpr (kRegLine) {   // in registers (NETA / 32 points per lane), spectrum to z
                float2 v[NETA / 32];
#pragma unroll
                for (int j = 0; j < NETA / 32; ++j) {
                    const size_t i = (size_t)m * NETA + lane + 32 * j;
                    v[j] = make_float2(ga[i] - ma, gb[i] - mb);
                }
                warp_fft_core<NETA>(v, wf, lane);
#pragma unroll
                for (int j = 0; j < NETA / 32; ++j) z[warp_fft_out<NETA>(lane, j)] = v[j];
                __syncwarp();
            } else {
                for (int l = lane; l < NETA; l += 32)
                    z[l] = make_float2(ga[(size_t)m * NETA + l] - ma, gb[(size_t)m * NETA + l] - mb);
                __syncwarp();
                linefft::warp_fft_line<NETA>(z, 1, tw);
            }
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane + 32 * j;
                if (k < H) {
                    const float2 zk = z[k], zn = z[(NETA - k) & (NETA - 1)];
                    // A = (Z[k] + conj Z[-k]) / 2, B = (Z[k] - conj Z[-k]) / (2i); acc += conj(A) B
                    const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
                    const float2 B = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
                    acc[j].x += A.x * B.x + A.y * B.y;
                    acc[j].y += A.x * B.y - A.y * B.x;
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < KPL; ++j) {
            const int k = lane + 32 * j;
            if (k < H) z[k] = acc[j];
        }
        __syncthreads();
        // C[k] over the warps in float64, extended by C[NETA - k] = conj C[k]; inverse transform by warp 0.
        // The correlation's scale does not move its argmax or parabolic offset, so it is not normalised.
        if (w == 0) {
            for (int k = lane; k < H; k += 32) {
                float cr = 0.f, ci = 0.f;   // eight FP32 partials (FP64 here kept GB300's narrow FP64 pipe busy)
                for (int v = 0; v < kEtaWarps; ++v) { cr += line[v][k].x; ci += line[v][k].y; }
                zc[k] = make_float2(cr, ci);
                if (k > 0 && k < NETA / 2) zc[NETA - k] = make_float2(cr, -ci);
            }
            __syncwarp();
            if constexpr (kRegLine) {
                WarpFftTw<NETA> wi;
                wi.load(twi, lane);
                float2 v[NETA / 32];
#pragma unroll
                for (int j = 0; j < NETA / 32; ++j) v[j] = zc[lane + 32 * j];
                warp_fft_core<NETA>(v, wi, lane);
#pragma unroll
                for (int j = 0; j < NETA / 32; ++j) cfin[warp_fft_out<NETA>(lane, j)] = v[j].x;
            } else {
                linefft::warp_fft_line<NETA>(zc, 1, twi);
                for (int d = lane; d < NETA; d += 32) cfin[d] = zc[d].x;
            }
            __syncwarp();
            // argmax over the shifts (the lowest shift among equal maxima), then the parabola
            int best = lane;
            for (int D = lane + 32; D < NETA; D += 32)
                if (cfin[D] > cfin[best]) best = D;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                if (cfin[ob] > cfin[best] || (cfin[ob] == cfin[best] && ob < best)) best = ob;
            }
            if (lane == 0) {
                const float off = parabola(cfin[(best + NETA - 1) % NETA], cfin[best], cfin[(best + 1) % NETA]);
                wshift[b] = (double)(best < NETA / 2 ? best : best - NETA) + off;
            }
        }
        __syncthreads();   // line, zc and cfin are reused by the next window
    }
    if (tid == 0) {
        // median of the window shifts (mean of the middle two for an even count)
        for (int i = 1; i < windows; ++i)
            for (int j = i; j > 0 && wshift[j] < wshift[j - 1]; --j) {
                const double t = wshift[j];
                wshift[j] = wshift[j - 1];
                wshift[j - 1] = t;
            }
        const double deta = windows % 2 ? wshift[windows / 2] : 0.5 * (wshift[windows / 2 - 1] + wshift[windows / 2]);
        const double tz = 2.0 * XCF_PI * deta / NETA;
        double s, c;
        sincos(0.5 * tz, &s, &c);
        const Q Rz = {c, 0.0, 0.0, s};
        const Q q0 = qload(q0s + 4 * (size_t)p);
        const Q q2 = rotate_in_detector(qload(q1s + 4 * (size_t)p), Rz, alpha);
        double dot = fabs(q2.w * q0.w + q2.x * q0.x + q2.y * q0.y + q2.z * q0.z);
        dot = fmin(dot, 1.0);
        const double upd = 2.0 * acos(dot) * 180.0 / XCF_PI;
        qstore(q_out + 4 * (size_t)p, q2);
        iters[p] += 1;
        if (upd < tol_deg) active[p] = 0;
    }
}

__global__ void k_update_xy(const double *__restrict__ qs, const float *__restrict__ shift,
                            const double *__restrict__ pcs, double pcz_def, int W, double alpha,
                            const int *__restrict__ active, int P, double *__restrict__ q1s) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !active[p]) return;
    const double L = (pcs ? pcs[3 * (size_t)p + 2] : pcz_def) * W;
    const double tx = atan((double)shift[2 * p + 1] / L), ty = atan((double)shift[2 * p] / L);
    double sx, cx, sy, cy;
    sincos(0.5 * tx, &sx, &cx);
    sincos(0.5 * ty, &sy, &cy);
    const Q R = qmul(Q{cx, sx, 0.0, 0.0}, Q{cy, 0.0, sy, 0.0});
    qstore(q1s + 4 * (size_t)p, rotate_in_detector(qload(qs + 4 * (size_t)p), R, alpha));
}

// per-pattern pattern centre: a change of (pcx, pcy) translates the gnomonic
// screen content by (dpcx W, dpcy H) px, so that part of the measured shift is
// the pattern centre's and the rest the orientation's
__global__ void k_shift_pc(const double *__restrict__ pcs, double pcx, double pcy, int W, int H,
                           const int *__restrict__ best, int P, float *__restrict__ shift) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || best[p] < 0) return;
    shift[2 * (size_t)p] = (float)((double)shift[2 * (size_t)p] - (pcs[3 * (size_t)p] - pcx) * W);
    shift[2 * (size_t)p + 1] = (float)((double)shift[2 * (size_t)p + 1] - (pcs[3 * (size_t)p + 1] - pcy) * H);
}

__global__ void k_gather_seeds(const double *__restrict__ lib_quats, const int *__restrict__ best, int P,
                               double *__restrict__ seeds) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int t = best[p];
    for (int k = 0; k < 4; ++k) seeds[4 * (size_t)p + k] = t >= 0 ? lib_quats[4 * (size_t)t + k] : (k == 0 ? 1.0 : 0.0);
}

__global__ void k_init_refine(const int *__restrict__ degen, const int *__restrict__ select, int P,
                              int *__restrict__ active, int *__restrict__ iters, float *__restrict__ peak) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    if (select && !select[p]) {   // not refined: outputs left as they are
        active[p] = 0;
        return;
    }
    active[p] = degen[p] ? 0 : 1;
    iters[p] = 0;
    peak[p] = 0.f;
}

// the 24 proper rotations of the cubic group 432, (w, x, y, z)
__constant__ double c_cubic[24][4] = {
    {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1},
    {0.70710678118654752440, 0.70710678118654752440, 0, 0}, {0.70710678118654752440, -0.70710678118654752440, 0, 0},
    {0.70710678118654752440, 0, 0.70710678118654752440, 0}, {0.70710678118654752440, 0, -0.70710678118654752440, 0},
    {0.70710678118654752440, 0, 0, 0.70710678118654752440}, {0.70710678118654752440, 0, 0, -0.70710678118654752440},
    {0.5, 0.5, 0.5, 0.5}, {0.5, 0.5, 0.5, -0.5}, {0.5, 0.5, -0.5, 0.5}, {0.5, 0.5, -0.5, -0.5},
    {0.5, -0.5, 0.5, 0.5}, {0.5, -0.5, 0.5, -0.5}, {0.5, -0.5, -0.5, 0.5}, {0.5, -0.5, -0.5, -0.5},
    {0, 0.70710678118654752440, 0.70710678118654752440, 0}, {0, 0.70710678118654752440, -0.70710678118654752440, 0},
    {0, 0.70710678118654752440, 0, 0.70710678118654752440}, {0, 0.70710678118654752440, 0, -0.70710678118654752440},
    {0, 0, 0.70710678118654752440, 0.70710678118654752440}, {0, 0, 0.70710678118654752440, -0.70710678118654752440},
};

__global__ void k_disorientation(const double *__restrict__ qa, const double *__restrict__ qb, int n,
                                 double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Q m = qmul(qload(qa + 4 * (size_t)i), qconj(qload(qb + 4 * (size_t)i)));
    const double nm = sqrt(m.w * m.w + m.x * m.x + m.y * m.y + m.z * m.z);
    double best = 0.0;
    for (int k = 0; k < 24; ++k) {
        const double w = c_cubic[k][0] * m.w - c_cubic[k][1] * m.x - c_cubic[k][2] * m.y - c_cubic[k][3] * m.z;
        best = fmax(best, fabs(w) / nm);
    }
    out[i] = 2.0 * acos(fmin(best, 1.0)) * 180.0 / XCF_PI;
}

// orientations and PCs of the rotation experiment (sampling-frequency
// section): entry 0 the reference (q, pc_ref), entry 1 + a L + j the crystal
// rotated by theta_j = (j - h) step about detector axis a, at pc_test
__global__ void k_scan_setup(const double *__restrict__ q, const double *__restrict__ pc_test, double pcx,
                             double pcy, double pcz, int h, double step_rad, double alpha, double *__restrict__ qs,
                             double *__restrict__ pcs) {
    const int L = 2 * h + 1, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > 3 * L) return;
    const Q q0 = qload(q);
    double *pc = pcs + 3 * (size_t)i;
    if (i == 0) {
        qstore(qs, qcanon(q0));
        pc[0] = pcx; pc[1] = pcy; pc[2] = pcz;
        return;
    }
    const int a = (i - 1) / L, j = (i - 1) % L;
    double s, c;
    sincos(0.5 * (j - h) * step_rad, &s, &c);
    const Q R = {c, a == 0 ? s : 0.0, a == 1 ? s : 0.0, a == 2 ? s : 0.0};
    qstore(qs + 4 * (size_t)i, rotate_in_detector(q0, R, alpha));
    if (pc_test) {
        pc[0] = pc_test[0]; pc[1] = pc_test[1]; pc[2] = pc_test[2];
    } else {
        pc[0] = pcx; pc[1] = pcy; pc[2] = pcz;
    }
}

}  // namespace

cudaError_t launch_project(const float *master, int M, const double *quats, const double *pcs,
                           const int *active, int P, const ProjArgs &a, float *out, cudaStream_t st) {
    ProjArgs b = a;   // the rotation's cosine and sine once, on the host
    b.ca = cos(a.alpha);
    b.sa = sin(a.alpha);
    if (P <= 0) return cudaSuccess;
    const size_t npx = (size_t)a.nx * a.ny;
    for (int p0 = 0; p0 < P; p0 += 65535) {          // grid.y limit
        const int np = P - p0 < 65535 ? P - p0 : 65535;
        // 16 pixels per thread: the per-block float64 frame set-up is amortised over 4096 pixels
        dim3 grid((unsigned)((npx + 4095) / 4096), np);
        k_project<<<grid, 256, 0, st>>>(master, M, quats + 4 * (size_t)p0, pcs ? pcs + 3 * (size_t)p0 : nullptr,
                                        active ? active + p0 : nullptr, b, out + npx * p0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_logpolar(const float *spatial, const int *active, int P, int N, int nr, int neta,
                            float rmin, float rmax, float *out, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (N <= kLpSmemSide && N % 2 == 0 && !(reinterpret_cast<uintptr_t>(spatial) & 15)) {
        const int sm = (int)(sizeof(float) * N * N);
        cudaError_t e = cudaFuncSetAttribute(k_logpolar_img, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float) * kLpSmemSide * kLpSmemSide));
        if (e != cudaSuccess) return e;
        k_logpolar_img<<<P, 256, sm, st>>>(spatial, active, N, nr, neta, rmin, rmax, out);
        return cudaGetLastError();
    }
    constexpr int kChunk = 65535 * kLpPats;          // grid.y limit
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        dim3 grid((nr * neta + 255) / 256, (np + kLpPats - 1) / kLpPats);
        k_logpolar<<<grid, 256, 0, st>>>(spatial + (size_t)N * N * p0, active ? active + p0 : nullptr, np, N, nr,
                                         neta, rmin, rmax, out + (size_t)nr * neta * p0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_update_xy(const double *q, const float *shift, const double *pcs, double pcz_def,
                             int W, double alpha, const int *active, int P, double *q1,
                             cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_update_xy<<<(P + 127) / 128, 128, 0, st>>>(q, shift, pcs, pcz_def, W, alpha, active, P, q1);
    return cudaGetLastError();
}

cudaError_t launch_eta_update(const float *lpT, const float *lpP, int nr, int neta, int windows,
                              const double *q0, const double *q1, double alpha, double tol_deg, int *active,
                              int *iters, double *q_out, int P, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (windows < 1 || windows > kMaxLpWindows || windows > nr) return cudaErrorInvalidValue;
#define XCF_ETA_CASE(NE)                                                                                    \
    case NE:                                                                                                \
        k_eta_update<NE><<<P, kEtaThreads, 0, st>>>(lpT, lpP, nr, windows, q0, q1, alpha, tol_deg, active,   \
                                                    iters, q_out);                                          \
        break;
    switch (neta) {
        XCF_ETA_CASE(32)
        XCF_ETA_CASE(64)
        XCF_ETA_CASE(128)
        XCF_ETA_CASE(256)
        XCF_ETA_CASE(512)
        default: return cudaErrorInvalidValue;   // neta = 2N for N = 16 .. 256
    }
#undef XCF_ETA_CASE
    return cudaGetLastError();
}

cudaError_t launch_gather_seeds(const double *lib_quats, const int *best, int P, double *seeds,
                                cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_gather_seeds<<<(P + 127) / 128, 128, 0, st>>>(lib_quats, best, P, seeds);
    return cudaGetLastError();
}

cudaError_t launch_shift_pc(const double *pcs, double pcx, double pcy, int W, int H, const int *best, int P,
                            float *shift, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_shift_pc<<<(P + 127) / 128, 128, 0, st>>>(pcs, pcx, pcy, W, H, best, P, shift);
    return cudaGetLastError();
}

cudaError_t launch_init_refine(const int *degen, const int *select, int P, int *active, int *iters, float *peak,
                               cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k_init_refine<<<(P + 127) / 128, 128, 0, st>>>(degen, select, P, active, iters, peak);
    return cudaGetLastError();
}

cudaError_t launch_disorientation(const double *qa, const double *qb, int n, double *out,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_disorientation<<<(n + 127) / 128, 128, 0, st>>>(qa, qb, n, out);
    return cudaGetLastError();
}

cudaError_t launch_scan_setup(const double *q, const double *pc_test, double pcx, double pcy, double pcz, int h,
                              double step_rad, double alpha, double *qs, double *pcs, cudaStream_t st) {
    const int n = 3 * (2 * h + 1) + 1;
    k_scan_setup<<<(n + 127) / 128, 128, 0, st>>>(q, pc_test, pcx, pcy, pcz, h, step_rad, alpha, qs, pcs);
    return cudaGetLastError();
}
