// Shared-memory 2-D FFT machinery and the all-pairs search body for the
// sides other than the tuned 128 and 256 kernels (16 .. 160 px, native 96 and
// 160 included): register line FFTs for N = R x 32 >= 64, radix-2 butterflies
// in shared memory below; used by the kernels of k_generic.cu.
#pragma once
#include "common.cuh"

namespace gen {

constexpr int kThreads = 256;

// A unit of whole warps working on one item: threads t = 0 .. n-1 of the
// unit (the CTA's threads base .. base + n - 1), named barrier `id` (0: the
// whole CTA, __syncthreads) and a shared-memory region of its own.  The
// search bodies take one, so that a CTA can run one item on all its threads
// or several items side by side on groups of warps.
struct Grp {
    int t, n, id;
    float4 *smem;
    __device__ __forceinline__ void sync() const {
        if (id == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};
__device__ __forceinline__ Grp cta_group() {
    extern __shared__ float4 smem_raw[];
    return Grp{(int)threadIdx.x, (int)blockDim.x, 0, smem_raw};
}

// FFT (unscaled) of `nlines` lines of N points held in shared memory: point i
// of line l at buf[l * ls + i * es]; tw[k] = exp(SIGN 2 pi i k / N), k < N/2.
// One warp per line.  By default N >= 64 (R x 32 with R = 2^k, 3 or 5) runs
// warp_fft_reg (registers and shuffles, each lane's twiddles loaded once per
// call) and N < 64 radix-2 butterflies in shared memory; RADIX2 = true takes
// the shared-memory radix-2 butterflies at any power-of-two N.
// (The unit's warps: w0 = its first warp index within the unit, nw warps.)
template <int N, bool RADIX2 = (N < 64)>
__device__ void smem_fft_lines(float2 *buf, int nlines, int ls, int es, const float2 *tw, int w0, int nw) {
    constexpr int LOG = cx_log2(N);
    const int lane = threadIdx.x & 31;
    if constexpr (!RADIX2) {   // N = R x 32 (R = 2^k, 3 or 5)
        WarpFftTw<N> t;
        t.load(tw, lane);
        for (int l = w0; l < nlines; l += nw) warp_fft_reg<N>(buf + l * ls, es, t, lane);
    } else {
        for (int l = w0; l < nlines; l += nw) {
            float2 *x = buf + l * ls;
            for (int i = lane; i < N; i += 32) {
                int j = __brev(i) >> (32 - LOG);
                if (i < j) {
                    float2 t = x[i * es];
                    x[i * es] = x[j * es];
                    x[j * es] = t;
                }
            }
            __syncwarp();
#pragma unroll 1
            for (int s = 0; s < LOG; ++s) {
                const int half = 1 << s;
                for (int b = lane; b < N / 2; b += 32) {
                    int k = b & (half - 1);
                    int i0 = ((b >> s) << (s + 1)) + k, i1 = i0 + half;
                    float2 w = tw[k << (LOG - 1 - s)];
                    float2 u = x[i0 * es], v = c_mul(x[i1 * es], w);
                    x[i0 * es] = c_add(u, v);
                    x[i1 * es] = c_sub(u, v);
                }
                __syncwarp();
            }
        }
    }
}

template <int N, bool RADIX2 = (N < 64)>
__device__ __forceinline__ void smem_fft_lines(float2 *buf, int nlines, int ls, int es, const float2 *tw) {
    smem_fft_lines<N, RADIX2>(buf, nlines, ls, es, tw, (int)(threadIdx.x >> 5), (int)(blockDim.x >> 5));
}

template <int N, bool RADIX2 = (N < 64)>
__device__ __forceinline__ void fft2_smem(float2 *buf, const float2 *tw, const Grp &g) {
    constexpr int LD = N + 1;
    smem_fft_lines<N, RADIX2>(buf, N, LD, 1, tw, g.t >> 5, g.n >> 5);   // rows
    g.sync();
    smem_fft_lines<N, RADIX2>(buf, N, 1, LD, tw, g.t >> 5, g.n >> 5);   // columns
    g.sync();
}
template <int N, bool RADIX2 = (N < 64)>
__device__ __forceinline__ void fft2_smem(float2 *buf, const float2 *tw) {
    fft2_smem<N, RADIX2>(buf, tw, cta_group());
}

template <int N>
__device__ void make_twiddles(float2 *tw, int sign, int t, int n) {
    for (int k = t; k < N / 2; k += n)
        tw[k] = make_float2(kTwTable<N>.re[k], sign > 0 ? kTwTable<N>.im[k] : -kTwTable<N>.im[k]);
}
template <int N>
__device__ void make_twiddles(float2 *tw, int sign) {
    make_twiddles<N>(tw, sign, (int)threadIdx.x, (int)blockDim.x);
}

// sum over the block of one FP32 partial per thread: warp sums in FP32, the
// warps' sums added in FP64 (keeps the hot loops off the FP64 pipe)
__device__ inline double block_sum_f(float v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += sh[i];
        sh[32] = s;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// max over the unit of one value per thread (sh: 33 floats of the unit's own)
__device__ inline float block_max(float v, float *sh, const Grp &g) {
    const int lane = g.t & 31, w = g.t >> 5, nw = g.n >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[w] = v;
    g.sync();
    if (w == 0) {
        v = lane < nw ? sh[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[32] = v;
    }
    g.sync();
    float r = sh[32];
    g.sync();
    return r;
}
__device__ inline float block_max(float v, float *sh) { return block_max(v, sh, cta_group()); }

// Z = X1 + i X2 over the full N x N spectrum, X_j = conj(St_j) Sp extended
// from the stored half (columns 0..N/2) by Hermitian symmetry.
template <int N>
__device__ __forceinline__ void build_pair_spectrum(float2 *buf, const float2 *__restrict__ t1,
                                                    const float2 *__restrict__ t2,
                                                    const float2 *__restrict__ sp, int t0, int nt) {
    constexpr int LD = N + 1, HW = N / 2 + 1;
    // each stored value (u, v <= N/2) gives Z(u, v) = X1 + i X2 and, for
    // 0 < v < N/2, Z(-u, -v) = conj X1 + i conj X2
    for (int k = t0; k < N * HW; k += nt) {
        const int u = k / HW, v = k - u * HW;
        const float2 s = sp[k];
        const float2 x1 = c_mulcj(t1[k], s), x2 = c_mulcj(t2[k], s);
        buf[u * LD + v] = make_float2(x1.x - x2.y, x1.y + x2.x);
        if (v > 0 && v < N / 2) buf[(u == 0 ? 0 : N - u) * LD + (N - v)] = make_float2(x1.x + x2.y, -x1.y + x2.x);
    }
}

// Z = X1 + i X2 at the N/32 points c = lane + 32 j of row r (build_pair_spectrum
// for one row, into registers).  The two halves of the row differ only in the
// stored row they read and in signs, so both are loaded through one index.
// Split in two so that a row's loads can be issued a row ahead: pair_row_load
// fetches the spectra, pair_row_make combines them.
template <int N>
struct PairRowRaw {
    float2 a[N / 32], b[N / 32], s[N / 32];
};
template <int N>
__device__ __forceinline__ void pair_row_load(PairRowRaw<N> &w, int r, int lane, const float2 *__restrict__ t1,
                                              const float2 *__restrict__ t2, const float2 *__restrict__ sp) {
    constexpr int HW = N / 2 + 1;
    const int rr = r == 0 ? 0 : N - r;
#pragma unroll
    for (int j = 0; j < N / 32; ++j) {
        const int c = lane + 32 * j;
        const int k = c <= N / 2 ? r * HW + c : rr * HW + (N - c);
        w.s[j] = sp[k];
        w.a[j] = t1[k];
        w.b[j] = t2[k];
    }
}
template <int N>
__device__ __forceinline__ void pair_row_make(float2 (&v)[N / 32], const PairRowRaw<N> &w, int lane) {
#pragma unroll
    for (int j = 0; j < N / 32; ++j) {
        const int c = lane + 32 * j;
        const float2 x1 = c_mulcj(w.a[j], w.s[j]), x2 = c_mulcj(w.b[j], w.s[j]);
        v[j] = c <= N / 2 ? make_float2(x1.x - x2.y, x1.y + x2.x) : make_float2(x1.x + x2.y, x2.x - x1.y);
    }
}
template <int N>
__device__ __forceinline__ void pair_row(float2 (&v)[N / 32], int r, int lane, const float2 *__restrict__ t1,
                                         const float2 *__restrict__ t2, const float2 *__restrict__ sp) {
    PairRowRaw<N> w;
    pair_row_load<N>(w, r, lane, t1, t2, sp);
    pair_row_make<N>(v, w, lane);
}

// search_body for N = R x 32 >= 64: per template pair, each warp builds its
// rows of Z from the spectra straight into registers, transforms them
// (warp_fft_core) and stores them once; after one barrier each warp loads its
// columns, transforms them and keeps the running maxima of the real and
// imaginary parts in registers (the surface is never written back); after a
// second barrier thread 0 combines the warps' maxima.
// PF: fetch the next row's spectra a row ahead (R x 6 more registers per
// thread: for CTAs of at most 512 threads, whose register budget has room)
template <int N, bool PF = true>
__device__ void search_body_reg(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                                int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                                const int *__restrict__ cand, int kc, const Grp &g) {
    constexpr int LD = N + 1, HW = N / 2 + 1, R = N / 32;
    float2 *buf = reinterpret_cast<float2 *>(g.smem);
    float2 *twi = buf + N * LD;
    float2 *red = twi + N;   // 32 entries
    const int lane = g.t & 31, w = g.t >> 5, nw = g.n >> 5;
    make_twiddles<N>(twi, +1, g.t, g.n);
    g.sync();
    WarpFftTw<N> tw;
    tw.load(twi, lane);
    const float2 *sp = Sp + (size_t)p * N * HW;
    const int n = cand ? kc : T;
    float best_v = -INFINITY;
    int best_t = -1;
    for (int pi = pb; pi < pe; ++pi) {
        const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
        const int t1 = cand ? cand[(size_t)p * kc + j1] : j1;
        const int t2 = cand ? cand[(size_t)p * kc + j2] : j2;
        const float2 *s1 = St + (size_t)max(t1, 0) * N * HW, *s2 = St + (size_t)max(t2, 0) * N * HW;
        // rows (the previous pair's column reads ended at its second barrier); the
        // spectra of the warp's next row are fetched before this row is transformed,
        // so their L2 latency overlaps the transform
        if constexpr (PF) {
            PairRowRaw<N> raw;
            if (w < N) pair_row_load<N>(raw, w, lane, s1, s2, sp);
            for (int r = w; r < N; r += nw) {
                float2 v[R];
                pair_row_make<N>(v, raw, lane);
                if (r + nw < N) pair_row_load<N>(raw, r + nw, lane, s1, s2, sp);
                warp_fft_core<N>(v, tw, lane);
#pragma unroll
                for (int j = 0; j < R; ++j) buf[r * LD + warp_fft_out<N>(lane, j)] = v[j];
            }
        } else {
            for (int r = w; r < N; r += nw) {
                float2 v[R];
                pair_row<N>(v, r, lane, s1, s2, sp);
                warp_fft_core<N>(v, tw, lane);
#pragma unroll
                for (int j = 0; j < R; ++j) buf[r * LD + warp_fft_out<N>(lane, j)] = v[j];
            }
        }
        g.sync();
        // columns: maxima only
        float m1 = -INFINITY, m2 = -INFINITY;
        for (int c = w; c < N; c += nw) {
            float2 v[R];
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = buf[(lane + 32 * j) * LD + c];
            warp_fft_core<N>(v, tw, lane);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                m1 = fmaxf(m1, v[j].x);
                m2 = fmaxf(m2, v[j].y);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if (lane == 0) red[w] = make_float2(m1, m2);
        g.sync();
        if (g.t == 0) {
            m1 = red[0].x;
            m2 = red[0].y;
            for (int i = 1; i < nw; ++i) {
                m1 = fmaxf(m1, red[i].x);
                m2 = fmaxf(m2, red[i].y);
            }
            if (t1 < 0) m1 = -INFINITY;
            if (t2 < 0) m2 = -INFINITY;
            if (t1 >= 0 && (m1 > best_v || (m1 == best_v && t1 < best_t))) { best_v = m1; best_t = t1; }
            if (j2 != j1 && t2 >= 0 && (m2 > best_v || (m2 == best_v && t2 < best_t))) { best_v = m2; best_t = t2; }
            if (peaks_all) {
                peaks_all[(size_t)p * n + j1] = m1;
                if (j2 != j1) peaks_all[(size_t)p * n + j2] = m2;
            }
        }
    }
    if (g.t == 0 && best_t >= 0) atomicMax(keys + p, pack_key(best_v, best_t));
}
template <int N, bool PF = true>
__device__ void search_body_reg(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                                int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                                const int *__restrict__ cand, int kc) {
    search_body_reg<N, PF>(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc, cta_group());
}

// search body with the whole surface in shared memory: per template pair the
// full spectrum Z is built in shared memory, transformed by rows and by
// columns with radix-2 butterfly line FFTs in shared memory, and scanned for
// the maxima (any power-of-two N up to 64; blockDim-strided loops)
template <int N>
__device__ void search_body_smem(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                                 int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                                 const int *__restrict__ cand, int kc, const Grp &g) {
    constexpr int LD = N + 1, HW = N / 2 + 1;
    float2 *buf = reinterpret_cast<float2 *>(g.smem);
    float2 *twi = buf + N * LD;
    float *redf = reinterpret_cast<float *>(twi + N);   // 33 entries
    make_twiddles<N>(twi, +1, g.t, g.n);
    const float2 *sp = Sp + (size_t)p * N * HW;
    // slots: every template, or this pattern's candidate list (entries < 0 are empty)
    const int n = cand ? kc : T;
    float best_v = -INFINITY;
    int best_t = -1;
    for (int pi = pb; pi < pe; ++pi) {
        const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
        const int t1 = cand ? cand[(size_t)p * kc + j1] : j1;
        const int t2 = cand ? cand[(size_t)p * kc + j2] : j2;
        g.sync();
        build_pair_spectrum<N>(buf, St + (size_t)max(t1, 0) * N * HW, St + (size_t)max(t2, 0) * N * HW, sp, g.t,
                               g.n);
        g.sync();
        fft2_smem<N, true>(buf, twi, g);
        float m1 = -INFINITY, m2 = -INFINITY;
        for (int idx = g.t; idx < N * N; idx += g.n) {
            float2 z = buf[(idx / N) * LD + idx % N];
            m1 = fmaxf(m1, z.x);
            m2 = fmaxf(m2, z.y);
        }
        m1 = block_max(m1, redf, g);
        m2 = block_max(m2, redf, g);
        if (t1 < 0) m1 = -INFINITY;
        if (t2 < 0) m2 = -INFINITY;
        if (t1 >= 0 && (m1 > best_v || (m1 == best_v && t1 < best_t))) { best_v = m1; best_t = t1; }
        if (j2 != j1 && t2 >= 0 && (m2 > best_v || (m2 == best_v && t2 < best_t))) { best_v = m2; best_t = t2; }
        if (peaks_all && g.t == 0) {
            peaks_all[(size_t)p * n + j1] = m1;
            if (j2 != j1) peaks_all[(size_t)p * n + j2] = m2;
        }
    }
    if (g.t == 0 && best_t >= 0) atomicMax(keys + p, pack_key(best_v, best_t));
}
template <int N>
__device__ void search_body_smem(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                                 int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                                 const int *__restrict__ cand, int kc) {
    search_body_smem<N>(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc, cta_group());
}

// One work item: pattern p against slot pairs [pb, pe) (slots = all
// templates, or the pattern's candidate list); smem_bytes<N>() of dynamic
// shared memory; folds the item's best into keys[p].  N >= 64 takes
// search_body_reg, smaller sides search_body_smem.
template <int N, bool PF = true>
__device__ void search_body(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                            int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                            const int *__restrict__ cand, int kc) {
    if constexpr (N >= 64)
        search_body_reg<N, PF>(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc);
    else
        search_body_smem<N>(St, T, Sp, p, pb, pe, keys, peaks_all, cand, kc);
}

// dynamic shared memory of one search item: the N x (N + 1) surface, N
// twiddles and the 34-entry reduction buffer
template <int N>
constexpr size_t smem_bytes() { return sizeof(float2) * ((size_t)N * (N + 1) + N + 34); }

}  // namespace gen
