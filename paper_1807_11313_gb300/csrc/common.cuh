// Shared device helpers of the ebsdxcf CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#define XCF_PI 3.14159265358979323846

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 c_mulcj(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by +i / -i
__device__ __forceinline__ float2 c_mul_pi(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 c_mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// ---------------------------------------------------- compile-time twiddles
// cos / sin of 2 pi k / n evaluated at compile time by Taylor series after
// exact range reduction (k mod n), so every constant below is a literal.
__host__ __device__ constexpr double cx_taylor_sin(double x) {
    double term = x, sum = x;
    for (int i = 1; i < 30; ++i) {
        term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double cx_taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 30; ++i) {
        term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        sum += term;
    }
    return sum;
}
// angle 2 pi k / n reduced to [-pi, pi]
__host__ __device__ constexpr double cx_angle(long k, long n) {
    long r = ((k % n) + n) % n;
    if (2 * r > n) r -= n;
    return 2.0 * XCF_PI * (double)r / (double)n;
}
template <long K, long N, int SIGN>
struct Tw {
    static constexpr double a = cx_angle(K, N);
    static constexpr float re = (float)cx_taylor_cos(a);
    static constexpr float im = (float)(SIGN * cx_taylor_sin(a));
};

// cos / sin of 2 pi k / N, k < N/2, as a table built at compile time (the
// Taylor series above after exact range reduction: correctly rounded to
// float), so that kernels fill their twiddle tables without FP64 work
template <int N>
struct TwTable {
    float re[N / 2], im[N / 2];
};
template <int N>
constexpr TwTable<N> make_tw_table() {
    TwTable<N> t{};
    for (int k = 0; k < N / 2; ++k) {
        const double a = cx_angle(k, N);
        t.re[k] = (float)cx_taylor_cos(a);
        t.im[k] = (float)cx_taylor_sin(a);
    }
    return t;
}
template <int N>
__device__ const TwTable<N> kTwTable = make_tw_table<N>();

// x * exp(SIGN 2 pi i K / N) with the trivial cases written out
template <long K, long N, int SIGN>
__device__ __forceinline__ float2 tw_mul(float2 x) {
    constexpr long r = ((K % N) + N) % N;
    if constexpr (r == 0) {
        return x;
    } else if constexpr (4 * r == N) {
        return SIGN > 0 ? c_mul_pi(x) : c_mul_mi(x);
    } else if constexpr (2 * r == N) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (4 * r == 3 * N) {
        return SIGN > 0 ? c_mul_mi(x) : c_mul_pi(x);
    } else if constexpr (8 * r == N || 8 * r == 3 * N || 8 * r == 5 * N || 8 * r == 7 * N) {
        // (+-1 +- i)/sqrt(2): two multiplies, two adds
        constexpr float h = 0.70710678118654752440f;
        constexpr float cr = Tw<K, N, SIGN>::re, ci = Tw<K, N, SIGN>::im;
        float s = (cr > 0 ? 1.f : -1.f), t = (ci > 0 ? 1.f : -1.f);
        // (x.x + i x.y)(s + i t) h
        return make_float2(h * (s * x.x - t * x.y), h * (s * x.y + t * x.x));
    } else {
        constexpr float cr = Tw<K, N, SIGN>::re, ci = Tw<K, N, SIGN>::im;
        return make_float2(fmaf(x.x, cr, -x.y * ci), fmaf(x.x, ci, x.y * cr));
    }
}

// ------------------------------------------------------------ static_for
template <int I, int E>
struct StaticFor {
    template <class F>
    __device__ __forceinline__ static void run(F &&f) {
        if constexpr (I < E) {
            f(std::integral_constant<int, I>{});
            StaticFor<I + 1, E>::run(f);
        }
    }
};

__host__ __device__ constexpr int cx_log2(int n) { return n <= 1 ? 0 : 1 + cx_log2(n / 2); }
__host__ __device__ constexpr int cx_bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// In-register radix-2 decimation-in-frequency FFT of R points,
// x[j] <- sum_i x[i] exp(SIGN 2 pi i i j / R) (unscaled).  Input in natural
// order, output in bit-reversed order: after the call x[p] holds X[bitrev(p)].
template <int R, int SIGN>
__device__ __forceinline__ void fft_reg_dif(float2 (&x)[R]) {
    constexpr int LOG = cx_log2(R);
    StaticFor<0, LOG>::run([&](auto stage) {
        constexpr int span = R >> (decltype(stage)::value + 1);
        StaticFor<0, R / (2 * span)>::run([&](auto blk) {
            StaticFor<0, span>::run([&](auto k) {
                constexpr int kk = decltype(k)::value;
                constexpr int i0 = decltype(blk)::value * 2 * span + kk;
                constexpr int i1 = i0 + span;
                float2 a = x[i0], b = x[i1];
                x[i0] = c_add(a, b);
                x[i1] = tw_mul<kk, 2 * span, SIGN>(c_sub(a, b));
            });
        });
    });
}

// ---------------------------------------------------- warp line FFT (N >= 64)
// One line of N = R x 32 points in shared memory (point i at x[i * es]),
// transformed by one warp in registers: lane l holds points l + 32 j
// (j < R).  R a power of two: decimation in frequency, the stages of span
// >= 32 pairing registers of a lane, the five of span < 32 pairing lanes
// through shuffles.  R = 3 or 5 (96- and 160-point lines): an R-point DFT
// over a lane's registers, the twiddles W_N^(l k1), then the same five
// shuffle stages for the 32-point DFT across lanes (Cooley-Tukey with N1 = R,
// N2 = 32).  The results go back in natural order (reversed-digit store
// addresses).  tw[k] = exp(SIGN 2 pi i k / N), k < N/2 (W^(k + N/2) = -W^k);
// WarpFftTw holds the twiddles one lane needs, so that a warp transforming
// several lines loads them once.
template <int N>
__device__ __forceinline__ float2 tw_any(const float2 *tw, int m) {   // W_N^m for 0 <= m < N
    const float2 w = tw[m < N / 2 ? m : m - N / 2];
    return m < N / 2 ? w : make_float2(-w.x, -w.y);
}

template <int N>
struct WarpFftTw {
    static constexpr int R = N / 32;
    static constexpr bool P2 = (R & (R - 1)) == 0;
    static constexpr int LR = P2 ? cx_log2(R) : 0;
    float2 wr[R > 1 ? R - 1 : 1];   // 2^k: register stage st (span 32 h'), pair (j, j + h'); else W_N^(l k1)
    float2 cr[P2 ? 1 : R - 1];      // R = 3, 5: W_R^m, m = 1 .. R-1
    float2 wc[4];                   // lane stage c < 4 (span 16 >> c): 1 on the upper lane of a pair
    __device__ __forceinline__ void load(const float2 *tw, int lane) {
        load_regs(tw, lane);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (!(lane & (16 >> c))) wc[c] = make_float2(1.f, 0.f);
    }
    __device__ __forceinline__ void load_regs(const float2 *tw, int lane) {
        if constexpr (P2) {
            int o = 0;
#pragma unroll
            for (int st = 0; st < LR; ++st) {
                const int hp = R >> (st + 1);
#pragma unroll
                for (int jm = 0; jm < hp; ++jm) wr[o + jm] = tw[(lane + 32 * jm) << st];
                o += hp;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) wc[c] = tw[(lane & ((16 >> c) - 1)) << (LR + c)];
        } else {
#pragma unroll
            for (int k1 = 1; k1 < R; ++k1) wr[k1 - 1] = tw_any<N>(tw, lane * k1);
#pragma unroll
            for (int m = 1; m < R; ++m) cr[m - 1] = tw_any<N>(tw, 32 * m);
#pragma unroll
            for (int c = 0; c < 4; ++c) wc[c] = tw_any<N>(tw, R * ((lane & ((16 >> c) - 1)) << c));
        }
    }
};

// The transform of warp_fft_reg on values already in registers: on entry
// v[j] = point lane + 32 j; on exit v[j] holds output warp_fft_out<N>(lane, j).
template <int N>
__device__ __forceinline__ void warp_fft_core(float2 (&v)[N / 32], const WarpFftTw<N> &t, int lane) {
    constexpr int R = N / 32;
    constexpr bool P2 = WarpFftTw<N>::P2;
    static_assert(N >= 64 && N % 32 == 0 && (P2 || R == 3 || R == 5), "line length R x 32, R = 2^k, 3 or 5");
    if constexpr (P2) {
        constexpr int LR = cx_log2(R);
        int o = 0;
#pragma unroll
        for (int st = 0; st < LR; ++st) {
            const int hp = R >> (st + 1);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (j & hp) continue;
                const float2 a = v[j], b = v[j + hp];
                v[j] = c_add(a, b);
                v[j + hp] = c_mul(c_sub(a, b), t.wr[o + (j & (hp - 1))]);
            }
            o += hp;
        }
    } else {
        float2 y[R];
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) {
            y[k1] = v[0];
#pragma unroll
            for (int j = 1; j < R; ++j) {
                const int m = (j * k1) % R;
                y[k1] = c_add(y[k1], m == 0 ? v[j] : c_mul(v[j], t.cr[m - 1]));
            }
        }
        v[0] = y[0];
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) v[k1] = c_mul(y[k1], t.wr[k1 - 1]);
    }
    // lane stages: the upper lane of a pair keeps p + v, the lower (p - v) W;
    // written as (p + sg v) wc with sg = +-1 and wc = 1 on the upper lane, so that no lane
    // evaluates both branches; the last stage's twiddle is 1 on every lane
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const int h = 16 >> c;
        const float sg = (lane & h) ? -1.f : 1.f;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const float2 p = make_float2(__shfl_xor_sync(0xffffffffu, v[j].x, h),
                                         __shfl_xor_sync(0xffffffffu, v[j].y, h));
            const float2 d = make_float2(fmaf(sg, v[j].x, p.x), fmaf(sg, v[j].y, p.y));
            v[j] = c < 4 ? c_mul(d, t.wc[c < 4 ? c : 0]) : d;
        }
    }
}

// output index held in v[j] of `lane` after warp_fft_core
template <int N>
__device__ __forceinline__ int warp_fft_out(int lane, int j) {
    constexpr int R = N / 32;
    if constexpr (WarpFftTw<N>::P2) {
        return __brev(lane + 32 * j) >> (32 - cx_log2(N));
    } else {
        return j + R * (__brev(lane) >> 27);   // the 32-point transform leaves lane order bit-reversed
    }
}

template <int N>
__device__ __forceinline__ void warp_fft_reg(float2 *x, int es, const WarpFftTw<N> &t, int lane) {
    constexpr int R = N / 32;
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = x[(lane + 32 * j) * es];
    warp_fft_core<N>(v, t, lane);
    // every lane has read its points (the shuffles joined the warp): write back in place
#pragma unroll
    for (int j = 0; j < R; ++j) x[warp_fft_out<N>(lane, j) * es] = v[j];
    __syncwarp();
}

// order-preserving float -> uint32 (larger float -> larger key)
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// key = (ordered peak << 32) | (0xffffffff - t): max key = highest peak,
// lowest template index on ties
__device__ __forceinline__ unsigned long long pack_key(float v, int t) {
    return ((unsigned long long)float_to_ordered(v) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)t);
}
