// The 128 x 128 all-pairs search as a device function (see k_search128.cu for
// the design), shared by the search kernel and the multi-map kernel.
#pragma once
#include "common.cuh"

namespace s128 {


constexpr int N = 128;
constexpr int HW = 65;          // stored columns of a half spectrum
constexpr int SPEC = N * HW;    // complex values per half spectrum
constexpr int NT = 512;
constexpr int NW = NT / 32;
constexpr int COL64 = 8192;     // offset of column 64 in the packed layout

// shared layout (float2 units)
constexpr int OFF_SP = 0;                  // pattern, packed layout, 8320
constexpr int OFF_BUF = SPEC;              // transpose buffer, 16384
constexpr int OFF_TW1 = OFF_BUF + N * N;   // W128^(l k2) at [l][k2], l < 8, k2 < 16
constexpr int OFF_TW2 = OFF_TW1 + 128;     // W128^(g k3) at [k3][g], k3 < 4, g < 32
constexpr int OFF_C64 = OFF_TW2 + 128;     // next pair's column 64: [2][128]
constexpr int OFF_RED = OFF_C64 + 256;     // [2][16 warps] (max re, max im)
constexpr int OFF_Y64 = OFF_RED + 2 * NW;  // column 64 of Z = X1 + i X2: [128]
constexpr int SMEM_F2 = OFF_Y64 + 128;
constexpr size_t SMEM_BYTES = sizeof(float2) * SMEM_F2;

// packed position of (row u, stored column q < 64): [u & 7][(u >> 3) / 2][q][(u >> 3) & 1]
__host__ __device__ __forceinline__ int pk(int u, int q) {
    const int l = u & 7, m = u >> 3;
    return (((l * 8 + (m >> 1)) * 64 + q) << 1) + (m & 1);
}

// round-1 output A[l][k2][v] (a warp stores 32 consecutive v of one (l, k2) and
// round 2 reads 32 consecutive v of one (l, k2): no swizzle needed)
__device__ __forceinline__ int idxA(int l, int k2, int v) { return ((l * 16 + k2) << 7) + v; }
// round-2 output B[row = 4 y + k3][g]: 16-byte pairs of g swizzled by row & 7 so
// that round 3's 16-byte loads (one row per thread) spread over every bank
__device__ __forceinline__ int idxB(int row, int g) {
    return (row << 5) + ((((g >> 1) ^ (row & 7)) << 1) | (g & 1));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// one radix-2 decimation-in-frequency stage (sign +) of an R-point register FFT
template <int R, int STAGE>
__device__ __forceinline__ void dif_stage(float2 (&x)[R]) {
    constexpr int span = R >> (STAGE + 1);
    StaticFor<0, R / (2 * span)>::run([&](auto blk) {
        StaticFor<0, span>::run([&](auto k) {
            constexpr int kk = decltype(k)::value;
            constexpr int i0 = decltype(blk)::value * 2 * span + kk;
            constexpr int i1 = i0 + span;
            const float2 a = x[i0], b = x[i1];
            x[i0] = c_add(a, b);
            x[i1] = tw_mul<kk, 2 * span, +1>(c_sub(a, b));
        });
    });
}

// stages 1..3 of a 32-point DIF FFT (stage 0 done by the caller) followed by
// the maxima of the real and the imaginary parts of its outputs: the last
// butterfly stage is folded into the maxima, max(a + b, a - b) = a + |b|
// (exact: rounding is monotonic)
__device__ __forceinline__ void fft32_rest_max(float2 (&x)[32], float &m1, float &m2) {
    dif_stage<32, 1>(x);
    dif_stage<32, 2>(x);
    dif_stage<32, 3>(x);
    m1 = x[0].x + fabsf(x[1].x);
    m2 = x[0].y + fabsf(x[1].y);
#pragma unroll
    for (int j = 2; j < 32; j += 2) {
        m1 = fmaxf(m1, x[j].x + fabsf(x[j + 1].x));
        m2 = fmaxf(m2, x[j].y + fabsf(x[j + 1].y));
    }
}

// exp(+2 pi i e / 128) from the compile-time table (e in [0, 128))
__device__ __forceinline__ float2 w128(int e) {
    const int r = e & 63;
    const float2 w = make_float2(kTwTable<N>.re[r], kTwTable<N>.im[r]);
    return e & 64 ? make_float2(-w.x, -w.y) : w;
}

// One work item of the search: pattern p against template pairs [pb, pe)
// (pairs (2i, 2i + 1); T odd pairs the last template with itself).  Runs on
// the calling CTA's NT threads and SMEM_BYTES of dynamic shared memory and
// folds the best (peak, template) of the item into keys[p].
__device__ __forceinline__ void search_body(const float2 *__restrict__ Spk, int T, const float2 *__restrict__ Sp,
                                            int p, int pb, int pe, unsigned long long *__restrict__ keys,
                                            float *__restrict__ peaks_all) {
    extern __shared__ float4 smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float2 *sp = sm + OFF_SP;
    float2 *buf = sm + OFF_BUF;
    float2 *tw1 = sm + OFF_TW1;
    float2 *tw2 = sm + OFF_TW2;
    float2 *c64 = sm + OFF_C64;
    float2 *red = sm + OFF_RED;
    float2 *y64 = sm + OFF_Y64;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // round-1 identity: warp -> sub-sequence l (rows u = l + 8 m), lane -> stored column q
    const int l1 = warp & 7;
    const int q = ((warp >> 3) << 5) + lane;
    // round-2 identity: warp -> k2, lane -> column residue g (columns g + 32 i)
    const int k2r = warp;
    const int g2 = lane;
    // round-3 identity: one row (y, k3) of B per thread

    // stage a template pair into shared memory with asynchronous copies: the
    // packed columns 0..63 of both templates (2 x 64 KB) fill the transpose
    // buffer exactly
    auto stage = [&](int pi) {
        const int t1 = 2 * pi, t2 = min(t1 + 1, T - 1);
        const float4 *s1 = reinterpret_cast<const float4 *>(Spk + (size_t)t1 * SPEC);
        const float4 *s2 = reinterpret_cast<const float4 *>(Spk + (size_t)t2 * SPEC);
        float4 *d = reinterpret_cast<float4 *>(buf);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cp_async16(d + k * NT + tid, s1 + k * NT + tid);
            cp_async16(d + 4096 + k * NT + tid, s2 + k * NT + tid);
        }
        cp_async_commit();
    };
    // column 64 of both templates of a pair, row u = tid < 128, copied by the
    // thread that turns it into y64[u] (so no barrier separates the two)
    auto stage64 = [&](int pi) {
        if (tid < 128) {
            const int t1 = 2 * pi, t2 = min(t1 + 1, T - 1);
            cp_async8(c64 + tid, Spk + (size_t)t1 * SPEC + COL64 + tid);
            cp_async8(c64 + 128 + tid, Spk + (size_t)t2 * SPEC + COL64 + tid);
        }
        cp_async_commit();
    };
    // column 64 of Z (self-conjugate: Z = X1 + i X2 directly), row u = tid
    auto make_y64 = [&]() {
        if (tid < 128) {
            const float2 s64 = sp[COL64 + tid];
            const float2 y1 = c_mulcj(c64[tid], s64), y2 = c_mulcj(c64[128 + tid], s64);
            y64[tid] = make_float2(y1.x - y2.y, y1.y + y2.x);
        }
    };

    {   // pattern spectrum (packed into shared memory) and twiddle tables
        const float2 *src = Sp + (size_t)p * SPEC;
        for (int i = tid; i < SPEC; i += NT) {
            const int u = i / HW, v = i % HW;
            sp[v < 64 ? pk(u, v) : COL64 + u] = src[i];
        }
        if (tid < 128) {
            tw1[tid] = w128((tid >> 4) * (tid & 15));          // [l][k2]
        } else if (tid < 256) {
            const int k3 = (tid - 128) >> 5, g = tid & 31;
            tw2[tid - 128] = w128(g * k3);                      // [k3][g]
        }
    }
    stage64(pb);
    stage(pb);
    cp_async_wait_all();
    __syncthreads();   // the pattern's column 64 is in place
    make_y64();

    float best_v = -INFINITY;
    int best_t = -1;

    // Per pair: each barrier only guards the writes into buf, so the register
    // FFT work of a round runs before the barrier that precedes its stores
    // and overlaps the other warps' shared-memory loads.
    for (int pi = pb; pi < pe; ++pi) {
        cp_async_wait_all();
        __syncthreads();   // buf holds pair pi, y64 its column 64; the previous round 3 is done with buf
        // reduce the previous pair's per-warp maxima
        if (pi > pb && tid == 0) {
            const float2 *rr = red + ((pi - 1) & 1) * NW;
            float m1 = rr[0].x, m2 = rr[0].y;
#pragma unroll
            for (int w = 1; w < NW; ++w) { m1 = fmaxf(m1, rr[w].x); m2 = fmaxf(m2, rr[w].y); }
            const int u1 = 2 * (pi - 1), u2 = min(u1 + 1, T - 1);
            if (m1 > best_v) { best_v = m1; best_t = u1; }
            if (u2 != u1 && m2 > best_v) { best_v = m2; best_t = u2; }
            if (peaks_all) {
                peaks_all[(size_t)p * T + u1] = m1;
                if (u2 != u1) peaks_all[(size_t)p * T + u2] = m2;
            }
        }

        // ---------------- round 1: 16-point column sub-FFTs ----------------
        float2 a[16], b[16];
        {
            const float4 *sp4 = reinterpret_cast<const float4 *>(sp) + (l1 * 8) * 64 + q;
            const float4 *tp4 = reinterpret_cast<const float4 *>(buf) + (l1 * 8) * 64 + q;
#pragma unroll
            for (int mp = 0; mp < 8; ++mp) {
                const float4 s4 = sp4[mp * 64];
                const float4 t1 = tp4[mp * 64], t2 = tp4[4096 + mp * 64];
                a[2 * mp] = c_mulcj(make_float2(t1.x, t1.y), make_float2(s4.x, s4.y));
                a[2 * mp + 1] = c_mulcj(make_float2(t1.z, t1.w), make_float2(s4.z, s4.w));
                b[2 * mp] = c_mulcj(make_float2(t2.x, t2.y), make_float2(s4.x, s4.y));
                b[2 * mp + 1] = c_mulcj(make_float2(t2.z, t2.w), make_float2(s4.z, s4.w));
            }
        }
        const bool q0 = q == 0;
        if (q0) {
            // columns 0 and 64 are self-conjugate: pack Z = X1 + i X2 directly
            // (column 0 from the products above, column 64 from y64)
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                a[m] = make_float2(a[m].x - b[m].y, a[m].y + b[m].x);
                b[m] = y64[l1 + 8 * m];
            }
        }
        fft_reg_dif<16, +1>(a);
        fft_reg_dif<16, +1>(b);
        __syncthreads();   // every thread has read the staged templates: buf is free
        {
            // second store: the conjugate-symmetric partner column (q > 0), or
            // column 64 (q = 0, whose b holds the column-64 transform)
            float2 *dst1 = buf + idxA(l1, 0, q);
            float2 *dst2 = buf + (q0 ? idxA(l1, 0, 64) : idxA((8 - l1) & 7, 0, 128 - q));
            const float4 *tw = reinterpret_cast<const float4 *>(tw1 + l1 * 16);
            StaticFor<0, 8>::run([&](auto kk) {
                constexpr int k2a = 2 * decltype(kk)::value;
                const float4 w2 = tw[k2a >> 1];
                StaticFor<0, 2>::run([&](auto ee) {
                    constexpr int k2 = k2a + decltype(ee)::value;
                    constexpr int P = cx_bitrev(k2, 4);
                    const float2 w = decltype(ee)::value ? make_float2(w2.z, w2.w) : make_float2(w2.x, w2.y);
                    const float2 fa = k2 ? c_mul(a[P], w) : a[P], fb = k2 ? c_mul(b[P], w) : b[P];
                    if (q0) {   // lane 0 of warps 0..7 only
                        dst1[k2 * 128] = fa;
                        dst2[k2 * 128] = fb;
                    } else {
                        dst1[k2 * 128] = make_float2(fa.x - fb.y, fa.y + fb.x);   // F1 + i F2
                        dst2[k2 * 128] = make_float2(fa.x + fb.y, fb.x - fa.y);   // conj(F1) + i conj(F2)
                    }
                });
            });
        }
        __syncthreads();

        // ------- round 2: radix 8 over l finishes the columns, radix 4 starts the rows -------
        float2 c[8][4];
#pragma unroll
        for (int l = 0; l < 8; ++l)
#pragma unroll
            for (int i = 0; i < 4; ++i) c[l][i] = buf[idxA(l, k2r, g2 + 32 * i)];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 t[8];
#pragma unroll
            for (int l = 0; l < 8; ++l) t[l] = c[l][i];
            fft_reg_dif<8, +1>(t);   // t[P] = C[k1 = bitrev3(P)]
#pragma unroll
            for (int P = 0; P < 8; ++P) c[P][i] = t[P];
        }
        if (pi + 1 < pe) stage64(pi + 1);   // c64 was last read for this pair's y64
        __syncthreads();   // every thread has read A: buf is free for B
        {
            const float2 w1 = tw2[32 + g2], w2 = tw2[64 + g2], w3 = tw2[96 + g2];
            StaticFor<0, 8>::run([&](auto pp) {
                constexpr int P = decltype(pp)::value;
                constexpr int k1 = cx_bitrev(P, 3);
                const int row = (k2r + 16 * k1) << 2;
                const float2 e0 = c[P][0], e1 = c[P][1], e2 = c[P][2], e3 = c[P][3];
                const float2 s02 = c_add(e0, e2), d02 = c_sub(e0, e2);
                const float2 s13 = c_add(e1, e3), d13 = c_mul_pi(c_sub(e1, e3));
                buf[idxB(row, g2)] = c_add(s02, s13);                          // k3 = 0
                buf[idxB(row + 1, g2)] = c_mul(c_add(d02, d13), w1);           // k3 = 1
                buf[idxB(row + 2, g2)] = c_mul(c_sub(s02, s13), w2);           // k3 = 2
                buf[idxB(row + 3, g2)] = c_mul(c_sub(d02, d13), w3);           // k3 = 3
            });
        }
        __syncthreads();

        // ------- round 3: 32-point row FFTs, max; the next pair streams into buf meanwhile -------
        float2 d[32];
        {
            const float4 *rowp = reinterpret_cast<const float4 *>(buf) + (tid << 4);
            const int sw = tid & 7;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 v = rowp[j ^ sw];
                d[2 * j] = make_float2(v.x, v.y);
                d[2 * j + 1] = make_float2(v.z, v.w);
            }
        }
        dif_stage<32, 0>(d);
        __syncthreads();   // every thread holds its row values: buf is free
        if (pi + 1 < pe) stage(pi + 1);
        float m1, m2;
        fft32_rest_max(d, m1, m2);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if (lane == 0) red[(pi & 1) * NW + warp] = make_float2(m1, m2);
        if (pi + 1 < pe) {   // the next pair's column 64 (all but the newest copy group have landed)
            cp_async_wait_one();
            make_y64();
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int pi = pe;
        const float2 *rr = red + ((pi - 1) & 1) * NW;
        float m1 = rr[0].x, m2 = rr[0].y;
#pragma unroll
        for (int w = 1; w < NW; ++w) { m1 = fmaxf(m1, rr[w].x); m2 = fmaxf(m2, rr[w].y); }
        const int u1 = 2 * (pi - 1), u2 = min(u1 + 1, T - 1);
        if (m1 > best_v) { best_v = m1; best_t = u1; }
        if (u2 != u1 && m2 > best_v) { best_v = m2; best_t = u2; }
        if (peaks_all) {
            peaks_all[(size_t)p * T + u1] = m1;
            if (u2 != u1) peaks_all[(size_t)p * T + u2] = m2;
        }
        atomicMax(keys + p, pack_key(best_v, best_t));
    }
}


}  // namespace s128
