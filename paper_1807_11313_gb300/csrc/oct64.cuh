// N = 64 search body on groups of eight lanes (the multi-map queue's
// XCF_BODY_OCT).
//
// Paper: the cross-correlation of Eqs. 3/6 and its maximum (Fig. 1 B-C) at
// the 64 x 64 crop of the FFT section (a 96 px detector cropped to 64).
//
// A 64-point line is 8 x 8: lane l of an eight-lane group holds the points
// l + 8 n1 (n1 < 8), transforms them with an 8-point FFT in registers,
// multiplies by W64^(l k1), transposes them through the group's buffer and
// finishes with a second 8-point FFT, after which it holds X[l + 8 k2].  The
// rows of Z = X1 + i X2 (two templates per complex inverse transform) are
// built from the spectra straight into registers, transformed and stored in
// the 64 x 64 surface buffer; after one barrier the columns are gathered,
// transformed and reduced to the two surfaces' maxima, the last butterfly
// stage folded into them.
//
// Bank layout: the four groups of a warp take lines 8 apart (deal), the
// surface buffer holds row r at column c ^ (r mod 8) ^ 8 ((r / 8) mod 2), and
// the transpose buffers have a row stride of 9 and start 72 entries apart:
// every shared-memory access of a warp takes two wavefronts, the least for
// its 256 bytes.
#pragma once
#include "common.cuh"
#include "generic.cuh"

namespace o64 {

constexpr int N = 64, HW = N / 2 + 1, SCR = 72;

// shared memory of one item on nt threads: surface, transpose buffers, warp maxima
__host__ __device__ constexpr size_t smem_bytes(int nt) {
    return sizeof(float2) * ((size_t)N * N + (size_t)(nt / 8) * SCR + 16);
}

// line (row or column) of the i-th (group, round): a warp's four groups 8 apart
__device__ __forceinline__ int deal(int i) {
    const int w = i >> 2, j = i & 3;
    return 32 * (w >> 3) + 8 * j + (w & 7);
}
__device__ __forceinline__ int zi(int r, int c) { return r * N + (c ^ (r & 7) ^ (((r >> 3) & 1) << 3)); }

// exp(+2 pi i e / 64), e in [0, 64)
__device__ __forceinline__ float2 w64(int e) {
    const int r = e & 31;
    const float2 w = make_float2(kTwTable<N>.re[r], kTwTable<N>.im[r]);
    return e & 32 ? make_float2(-w.x, -w.y) : w;
}

// decimation-in-frequency stages [S0, S1) of an 8-point transform (sign +)
template <int S0, int S1>
__device__ __forceinline__ void dif8(float2 (&x)[8]) {
    StaticFor<S0, S1>::run([&](auto stage) {
        constexpr int span = 8 >> (decltype(stage)::value + 1);
        StaticFor<0, 8 / (2 * span)>::run([&](auto blk) {
            StaticFor<0, span>::run([&](auto k) {
                constexpr int kk = decltype(k)::value;
                constexpr int i0 = decltype(blk)::value * 2 * span + kk;
                constexpr int i1 = i0 + span;
                const float2 a = x[i0], b = x[i1];
                x[i0] = c_add(a, b);
                x[i1] = tw_mul<kk, 2 * span, +1>(c_sub(a, b));
            });
        });
    });
}

// 64-point inverse DFT of a line held as a[n1] = x[8 n1 + l] by an eight-lane
// group (mask gm): on exit a[p] = X[l + 8 bitrev3(p)]; with FOLD the last
// stage (span 1, no twiddle) is left to the caller.  tw[j] = W64^(l (j + 1)).
template <bool FOLD>
__device__ __forceinline__ void line(float2 (&a)[8], const float2 (&tw)[7], float2 *scr, int l, unsigned gm) {
    dif8<0, 3>(a);   // a[p] = A[k1 = bitrev3(p)], A[k1] = sum_n1 x[8 n1 + l] W8^(n1 k1)
    StaticFor<0, 8>::run([&](auto pp) {
        constexpr int p = decltype(pp)::value;
        constexpr int k1 = cx_bitrev(p, 3);
        scr[9 * l + k1] = k1 == 0 ? a[p] : c_mul(a[p], tw[k1 - 1]);
    });
    __syncwarp(gm);
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) a[n2] = scr[9 * n2 + l];
    __syncwarp(gm);
    if (FOLD)
        dif8<0, 2>(a);
    else
        dif8<0, 3>(a);
}

// pattern p against template pairs [pb, pe) (slot indices into cand when
// cand != null) on the group g (a multiple of 32 threads, smem_bytes(g.n) of
// shared memory); folds the item's best (peak, template) into keys[p]
__device__ inline void search_body(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, int p, int pb,
                                   int pe, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
                                   const int *__restrict__ cand, int kc, const gen::Grp &g) {
    float2 *zb = reinterpret_cast<float2 *>(g.smem);
    float2 *red = zb + N * N + (g.n / 8) * SCR;   // one entry per warp
    const int lane = g.t & 31, l = g.t & 7, gi = g.t >> 3, ng = g.n >> 3, w = g.t >> 5, nw = g.n >> 5;
    float2 *scr = zb + N * N + gi * SCR;
    const unsigned gm = 0xffu << (lane & 24);
    float2 tw[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) tw[j] = w64((l * (j + 1)) & (N - 1));
    const float2 *sp = Sp + (size_t)p * N * HW;
    const int n = cand ? kc : T;
    float best_v = -INFINITY;
    int best_t = -1;
    for (int pi = pb; pi < pe; ++pi) {
        const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
        const int t1 = cand ? cand[(size_t)p * kc + j1] : j1;
        const int t2 = cand ? cand[(size_t)p * kc + j2] : j2;
        const float2 *s1 = St + (size_t)max(t1, 0) * N * HW, *s2 = St + (size_t)max(t2, 0) * N * HW;
        // rows: Z(r, l + 8 m) = (conj s1 + i conj s2) p at (r, l + 8 m) for m < 4,
        // and (s1 + i s2) conj p at (-r, 64 - l - 8 m) for m >= 4 (Hermitian
        // symmetry of both surfaces; it also serves lane 0's column 32)
        for (int i = gi; i < N; i += ng) {
            const int r = deal(i), rr = (N - r) & (N - 1);
            float2 a[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int k = m < 4 ? r * HW + l + 8 * m : rr * HW + (N - l - 8 * m);
                const float2 x1 = __ldg(s1 + k), x2 = __ldg(s2 + k), ps = __ldg(sp + k);
                a[m] = m < 4 ? c_mul(make_float2(x1.x + x2.y, x2.x - x1.y), ps)
                             : c_mulcj(ps, make_float2(x1.x - x2.y, x1.y + x2.x));
            }
            line<false>(a, tw, scr, l, gm);
#pragma unroll
            for (int q = 0; q < 8; ++q) zb[zi(r, l + 8 * cx_bitrev(q, 3))] = a[q];
        }
        g.sync();
        // columns: maxima only
        float m1 = -INFINITY, m2 = -INFINITY;
        for (int i = gi; i < N; i += ng) {
            const int c = deal(i);
            float2 a[8];
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) a[n1] = zb[zi(8 * n1 + l, c)];
            line<true>(a, tw, scr, l, gm);
            // max(a + b, a - b) = a + |b| per real component
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                m1 = fmaxf(m1, a[k].x + fabsf(a[k + 1].x));
                m2 = fmaxf(m2, a[k].y + fabsf(a[k + 1].y));
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if (lane == 0) red[w] = make_float2(m1, m2);
        g.sync();   // every column read: the next pair may write the surface
        if (g.t == 0) {
            m1 = red[0].x;
            m2 = red[0].y;
            for (int k = 1; k < nw; ++k) {
                m1 = fmaxf(m1, red[k].x);
                m2 = fmaxf(m2, red[k].y);
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

}  // namespace o64
