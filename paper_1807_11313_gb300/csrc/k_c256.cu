// 256 x 256 all-pairs search on thread-block clusters of four CTAs.
//
// Paper: the cross-correlation of Eqs. 3/6 (conj(S_t) S_p, inverse FFT, peak)
// for every template of the library (Fig. 1 B-C), at the 256 x 256 detector.
//
// The complex 256 x 256 array Z = X1 + i X2 of a template pair (two real
// surfaces per complex inverse FFT, as at the smaller sizes) is 512 KB: more
// than one SM's shared memory, so it lives in the distributed shared memory
// of a cluster.  CTA c owns 64 rows -- 32 pairs {u, -u}, so that the
// Hermitian half of every row it builds comes from rows it also owns -- and
// after the row transforms every CTA reads the 64 columns it owns from all
// four CTAs (ld.shared::cluster) and transforms them.  Only the per-surface
// maxima leave the cluster.
//
// A 256-point line transform runs on a 16-thread group: a 16-point FFT in
// registers, the 256-point twiddle, a transpose through a 2 KB XOR-swizzled
// shared buffer, a second 16-point FFT.  Rows are placed in their owner's
// buffer at column x ^ ((slot >> 1) & 15), which makes both the row-phase
// stores and the column-phase cluster loads free of bank conflicts.
//
// Every CTA of a cluster runs the same items, pairs and barriers (all bounds
// come from the cluster index and the kernel arguments), so the two cluster
// barriers per template pair always complete.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int N = 256, HW = N / 2 + 1, NC = 4, NT = 256;
constexpr int ROWS = N / NC;                      // rows (and columns) per CTA
constexpr size_t ZC_F2 = (size_t)ROWS * N;        // 128 KB of row-transformed data
constexpr size_t SCR_F2 = (NT / 16) * 256;        // one 16 x 16 transpose buffer per group

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float4 ld_cluster4(uint32_t addr) {   // 16-byte aligned
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
// arrive without release: for a barrier that orders reads already consumed
// before it against writes after it
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ float ld_cluster_f(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// cos and sin of 2 pi n / 16
__device__ constexpr float kW16c[16] = {Tw<0, 16, 1>::re,  Tw<1, 16, 1>::re,  Tw<2, 16, 1>::re,  Tw<3, 16, 1>::re,
                                        Tw<4, 16, 1>::re,  Tw<5, 16, 1>::re,  Tw<6, 16, 1>::re,  Tw<7, 16, 1>::re,
                                        Tw<8, 16, 1>::re,  Tw<9, 16, 1>::re,  Tw<10, 16, 1>::re, Tw<11, 16, 1>::re,
                                        Tw<12, 16, 1>::re, Tw<13, 16, 1>::re, Tw<14, 16, 1>::re, Tw<15, 16, 1>::re};
__device__ constexpr float kW16s[16] = {Tw<0, 16, 1>::im,  Tw<1, 16, 1>::im,  Tw<2, 16, 1>::im,  Tw<3, 16, 1>::im,
                                        Tw<4, 16, 1>::im,  Tw<5, 16, 1>::im,  Tw<6, 16, 1>::im,  Tw<7, 16, 1>::im,
                                        Tw<8, 16, 1>::im,  Tw<9, 16, 1>::im,  Tw<10, 16, 1>::im, Tw<11, 16, 1>::im,
                                        Tw<12, 16, 1>::im, Tw<13, 16, 1>::im, Tw<14, 16, 1>::im, Tw<15, 16, 1>::im};

// home of row u: owner CTA and slot.  Row classes {u, 256 - u}; class b (the
// smaller member, classes 0 and 128 merged into one pair {0, 128}) goes to
// CTA b / 32, slot 2 (b mod 32) for the member below 128, +1 for the other.
__device__ __forceinline__ void row_home(int u, int &owner, int &slot) {
    int b = u <= 128 ? u : N - u;
    const int second = u >= 128;
    if (b == 128) b = 0;
    owner = b >> 5;
    slot = 2 * (b & 31) + second;
}
__device__ __forceinline__ int zc_index(int slot, int x) { return slot * N + (x ^ ((slot >> 1) & 15)); }

// 256-point DFT (X[k] = sum_n x[n] e^{SIGN 2 pi i nk/256}) of a line held by
// a 16-thread group: on entry a[n1] = x[16 n1 + t]; on exit a[p] =
// X[t + 16 bitrev4(p)].  tw[k] = e^{+2 pi i t k / 256}; scr = the group's buffer.
template <int SIGN>
__device__ __forceinline__ void line_fft(float2 (&a)[16], const float2 (&tw)[16], float2 *scr, int t) {
    fft_reg_dif<16, SIGN>(a);   // a[p] = A[bitrev(p)], A[k1] = sum_n1 x[16 n1 + t] e^{SIGN 2 pi i n1 k1 / 16}
    StaticFor<0, 16>::run([&](auto pp) {
        constexpr int p = decltype(pp)::value;
        constexpr int k1 = cx_bitrev(p, 4);
        float2 w = tw[k1];
        if (SIGN < 0) w.y = -w.y;
        const float2 v = k1 == 0 ? a[p] : c_mul(a[p], w);
        scr[t * 16 + (k1 ^ t)] = v;
    });
    const unsigned gm = 0xffffu << (threadIdx.x & 16);   // the group's half of the warp
    __syncwarp(gm);
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) a[n2] = scr[n2 * 16 + (t ^ n2)];
    __syncwarp(gm);
    fft_reg_dif<16, SIGN>(a);   // a[p] = X[t + 16 bitrev(p)]
}
__device__ __forceinline__ void line_ifft(float2 (&a)[16], const float2 (&tw)[16], float2 *scr, int t) {
    line_fft<+1>(a, tw, scr, t);
}

// rows of Z = X1 + i X2 owned by CTA c, X_j = f_j conj(T_j) P_j (half spectra
// T_j, P_j extended by Hermitian symmetry), transformed along v into Zc.
// Group g builds and transforms the row pairs j = g and g + 16.
__device__ __forceinline__ void rows_phase(float2 *Zc, const float2 *__restrict__ s1, const float2 *__restrict__ p1,
                                           float f1, const float2 *__restrict__ s2, const float2 *__restrict__ p2,
                                           float f2, const float2 (&tw)[16], float2 *scr, int c, int g, int t) {
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
        const int j = g + 16 * (r >> 1), b = 32 * c + j;
        const int u0 = b, u1 = b == 0 ? 128 : N - b;
        const int u = (r & 1) ? u1 : u0;
        const int pu = (N - u) & (N - 1);
        float2 a[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const int v = 16 * n1 + t;
            const bool direct = v <= 128;
            const int k = direct ? u * HW + v : pu * HW + (N - v);   // Hermitian half: X(u, v) = conj(X(-u, 256 - v))
            float2 x1 = c_mulcj(__ldg(s1 + k), __ldg(p1 + k)), x2 = c_mulcj(__ldg(s2 + k), __ldg(p2 + k));
            x1 = make_float2(x1.x * f1, x1.y * f1);
            x2 = make_float2(x2.x * f2, x2.y * f2);
            a[n1] = direct ? make_float2(x1.x - x2.y, x1.y + x2.x) : make_float2(x1.x + x2.y, -x1.y + x2.x);
        }
        line_ifft(a, tw, scr, t);
        const int slot = 2 * j + (r & 1);
#pragma unroll
        for (int q = 0; q < 16; ++q) Zc[zc_index(slot, t + 16 * cx_bitrev(q, 4))] = a[q];
    }
}

// L2 prefetch of one quarter (this CTA's share) of a template's half spectrum:
// the four CTAs of a cluster together bring the whole spectrum into L2 ahead
// of the row phase that reads it
constexpr uint32_t kSpecBytes = (uint32_t)(N * HW * sizeof(float2));   // 264,192 B, a multiple of 64
__device__ __forceinline__ void prefetch_quarter(const float2 *spec, int c) {
    const char *base = reinterpret_cast<const char *>(spec) + (size_t)c * (kSpecBytes / NC);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base), "r"(kSpecBytes / NC) : "memory");
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------- search on 512-thread CTAs
// The same cluster search with 32 groups of 16 threads per CTA (sixteen warps
// per SM to hide the latency of the row loads and the cluster gathers).
//
// Rows are owned by residue class: CTA c holds every row u with u mod 16 in
// R_c (R_0 = {0, 8, 1, 15}, R_1 = {2, 14, 3, 13}, R_2 = {4, 12, 5, 11},
// R_3 = {6, 10, 7, 9}; each set is closed under negation mod 16), row
// u = r + 16 b at slot 16 i + b for r the i-th member of R_c.  A column
// transform's lane l gathers the rows l + 16 n1, all from one owner, at one
// base address plus constant offsets.  Rows sit at column x ^ 4 i, which keeps
// the two half-warps' gathers of columns x and x + 2 free of bank conflicts.
//
// A group builds a row u together with its conjugate row -u: lane l holds u
// at columns v = l + 16 m and -u at v = 16 - l + 16 m (m < 16, mod 256).  The
// lane loads the stored half spectra at (u, l + 16 m) and (-u, 16 - l + 16 m)
// for m < 8 (all within v <= 128), and each value gives an element of both
// rows: Z(u, v) = W p directly, and Z(-u, -v) = V conj(p) through the
// Hermitian symmetry X_j(-u, -v) = conj X_j(u, v) of the two real surfaces,
// where W = conj(s1) + i conj(s2) and V = s1 + i s2.  Lane 0's second row is
// held at columns 16 + 16 m (its last register is column 0), which the
// twiddle e^{+2 pi i 16 k1 / 256} of the first 16-point pass accounts for.
// CTA 0's rows 0 and 128 are each their own conjugate: one group builds row 0
// as the pair (0, 0), transforms and stores it, then row 128 as the pair
// (128, 128) in the same registers.
namespace cw {

constexpr int NT = 512, NG = NT / 16;
constexpr size_t ZC_F2 = (size_t)ROWS * N;         // 128 KB of row-transformed data
constexpr size_t SCR_F2 = (size_t)NG * 256;        // one 16 x 16 transpose buffer per group
constexpr size_t TW_F2 = 256;                      // [k1][l]: e^{+2 pi i l k1 / 256}
constexpr size_t SMEM_BYTES = (ZC_F2 + SCR_F2 + TW_F2) * sizeof(float2) + 64 * sizeof(float);

// search layout of a template's half spectrum: row u, piece (j < 4, group
// lam < 17) holds columns lam + 16 (2 j) and lam + 16 (2 j + 1) (group 16:
// columns 16 .. 128).  A lane's eight columns d + 16 m (d = l, or 16 - l for
// the conjugate row) are its group's four 16-byte pieces, and the 16 lanes
// of a group read 256 contiguous bytes per piece.
constexpr int PK_ROW = 4 * 17 * 2;              // float2 per row (1,088 bytes)
constexpr size_t PK_F2 = (size_t)N * PK_ROW;    // float2 per template
constexpr uint32_t kPackBytes = (uint32_t)(PK_F2 * sizeof(float2));
static_assert(kPackBytes % (16 * NC) == 0, "a quarter of a packed template is a whole number of 16-byte units");

// member i of R_c at 4 c + i, and its inverse (residue r -> 4 owner + i), as nibbles
constexpr int kClass[16] = {0, 8, 1, 15, 2, 14, 3, 13, 4, 12, 5, 11, 6, 10, 7, 9};
constexpr unsigned long long home_pack() {
    unsigned long long h = 0;
    for (int k = 0; k < 16; ++k) h |= (unsigned long long)k << (4 * kClass[k]);
    return h;
}
constexpr unsigned long long kHome = home_pack();
constexpr bool classes_closed() {   // every R_c closed under negation mod 16
    for (int k = 0; k < 16; ++k) {
        const int neg = (16 - kClass[k]) & 15;
        if ((int)((kHome >> (4 * neg)) & 15) >> 2 != k >> 2) return false;
    }
    return true;
}
static_assert(classes_closed(), "row classes of a CTA must be closed under negation");

__device__ __forceinline__ int slot_of(int u) {
    const int h = (int)((kHome >> (4 * (u & 15))) & 15);
    return 16 * (h & 3) + (u >> 4);
}
__device__ __forceinline__ int zc_at(int slot, int x) { return slot * N + (x ^ (4 * (slot >> 4))); }

// the two rows group g of CTA c builds (ub = -ua except for CTA 0's last group)
__device__ __forceinline__ void unit_rows(int c, int g, int &ua, int &ub) {
    if (c > 0) {
        ua = (g < 16 ? 2 * c : 2 * c + 1) + 16 * (g & 15);
    } else if (g < 16) {
        ua = 1 + 16 * g;
    } else if (g < 24) {
        ua = 8 + 16 * (g - 16);
    } else if (g < 31) {
        ua = 16 * (g - 23);
    } else {
        ua = 0;
    }
    ub = ua == 0 ? N / 2 : N - ua;
}

__device__ __forceinline__ void prefetch_packed(const float2 *spec, int c) {   // this CTA's quarter into L2
    const char *base = reinterpret_cast<const char *>(spec) + (size_t)c * (kPackBytes / NC);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base), "r"(kPackBytes / NC) : "memory");
}

// lane loads of one row at columns d + 16 m (m < 8), templates in the search
// layout, pattern in the plain one: x[m] = (conj s1 + i conj s2) p when
// DIRECT, y[15 - m] = (s1 + i s2) conj p
template <bool DIRECT>
__device__ __forceinline__ void build_half(const float2 *__restrict__ k1, const float2 *__restrict__ k2,
                                           const float2 *__restrict__ sp, int row, int d, float2 (&x)[16],
                                           float2 (&y)[16]) {
    const float4 *q1 = reinterpret_cast<const float4 *>(k1 + (size_t)row * PK_ROW) + d;
    const float4 *q2 = reinterpret_cast<const float4 *>(k2 + (size_t)row * PK_ROW) + d;
    const float2 *pp = sp + row * HW + d;
    auto emit = [&](int m, float ax, float ay, float bx, float by, float2 p) {
        if (DIRECT) x[m] = c_mul(make_float2(ax + by, bx - ay), p);
        y[15 - m] = c_mulcj(p, make_float2(ax - by, ay + bx));
    };
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 A = __ldg(q1 + 17 * j), B = __ldg(q2 + 17 * j);
        const float2 p0 = __ldg(pp + 32 * j), p1 = __ldg(pp + 32 * j + 16);
        emit(2 * j, A.x, A.y, B.x, B.y, p0);
        emit(2 * j + 1, A.z, A.w, B.z, B.w, p1);
    }
}

// the search layout of T half spectra (one-off, when the library is built)
__global__ void k_pack_c256(const float2 *__restrict__ src, int T, float2 *__restrict__ dst) {
    const size_t total = (size_t)T * PK_F2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t t = i / PK_F2;
        const int k = (int)(i - t * PK_F2), u = k / PK_ROW, r = k - u * PK_ROW;
        const int pc = r >> 1, j = pc / 17, lam = pc - 17 * j;
        dst[i] = src[t * (size_t)(N * HW) + (size_t)u * HW + lam + 16 * (2 * j + (r & 1))];
    }
}

// decimation-in-frequency stages [S0, S1) of a 16-point transform in registers
template <int S0, int S1, int SIGN>
__device__ __forceinline__ void dif16(float2 (&x)[16]) {
    StaticFor<S0, S1>::run([&](auto stage) {
        constexpr int span = 16 >> (decltype(stage)::value + 1);
        StaticFor<0, 16 / (2 * span)>::run([&](auto blk) {
            StaticFor<0, span>::run([&](auto k) {
                constexpr int kk = decltype(k)::value;
                constexpr int i0 = decltype(blk)::value * 2 * span + kk;
                constexpr int i1 = i0 + span;
                const float2 a = x[i0], b = x[i1];
                x[i0] = c_add(a, b);
                x[i1] = tw_mul<kk, 2 * span, SIGN>(c_sub(a, b));
            });
        });
    });
}

// first half of a 256-point inverse DFT on a 16-thread group: lane l holds
// x[n2 + 16 n1] in a[n1 - e] (e = 0, or 1 for a line started at column 16);
// the 16-point pass over n1, the twiddle w(k1) = e^{+2 pi i (n2 + 16 e) k1 / 256}
// and the transpose, after which a[n2'] = A[k1 = l][n2'] for the second pass
template <class TW>
__device__ __forceinline__ void ifft256_pass1(float2 (&a)[16], TW w, int n2, float2 *scr, int l) {
    dif16<0, 4, +1>(a);
    StaticFor<0, 16>::run([&](auto pp) {
        constexpr int p = decltype(pp)::value;
        constexpr int k1 = cx_bitrev(p, 4);
        scr[n2 * 16 + (k1 ^ n2)] = k1 == 0 ? a[p] : c_mul(a[p], w(k1));
    });
    const unsigned gm = 0xffffu << (threadIdx.x & 16);
    __syncwarp(gm);
#pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = scr[q * 16 + (l ^ q)];
    __syncwarp(gm);
}


}  // namespace cw

// pattern p, template pairs [pb, pe) (slot indices into cand when cand != null)
__global__ void __launch_bounds__(cw::NT, 1)
k_search_c256w(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, const int *__restrict__ degen,
               int nchunks, int ppc, int n_items, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
               const int *__restrict__ cand, int kc) {
    using namespace cw;
    extern __shared__ float4 smem_raw[];
    float2 *Zc = reinterpret_cast<float2 *>(smem_raw);
    float2 *scr_all = Zc + cw::ZC_F2;
    float2 *twa = scr_all + cw::SCR_F2;
    float *red = reinterpret_cast<float *>(twa + TW_F2);   // [0..15] warp maxima, [32..33] CTA maxima
    const int tid = threadIdx.x, l = tid & 15, g = tid >> 4, warp = tid >> 5, lane = tid & 31;
    const int c = (int)cluster_rank();
    const int cid = blockIdx.x / NC, ncl = gridDim.x / NC;
    float2 *scr = scr_all + g * 256;
    const int n = cand ? kc : T;
    bool pending = false;   // a column-phase barrier arrived on but not yet waited for
    const int npairs = (n + 1) / 2;

    for (int i = tid; i < 256; i += cw::NT) {   // twa[k1][l]
        const int ll = i & 15, k1 = i >> 4;
        double s, co;
        sincospi(2.0 * ll * k1 / N, &s, &co);
        twa[i] = make_float2((float)co, (float)s);
    }
    // row phase: this group's two rows, their slots; lane l's second row starts at column sg
    int ua, ub;
    unit_rows(c, g, ua, ub);
    const bool singles = ua == 0;   // rows 0 and 128 (ub), each its own conjugate
    const int sa = slot_of(ua), sb = slot_of(ub), sg = 16 - l, ng = sg & 15;
    // column phase: lane l's rows l + 16 n1 at owner o, slots 16 i + n1; columns 64 c + 2 g + q
    const int hm = (int)((kHome >> (4 * l)) & 15), io = hm & 3;
    const uint32_t zc_local = (uint32_t)__cvta_generic_to_shared(Zc);
    const uint32_t cbase = map_to_rank(zc_local, (uint32_t)(hm >> 2)) +
                           (uint32_t)((16 * io * N + ((ROWS * c + 2 * g) ^ (4 * io))) * sizeof(float2));
    const uint32_t red_local = (uint32_t)__cvta_generic_to_shared(red);
    __syncthreads();   // twa

    auto pair_templates = [&](int it, int pi, int &t1, int &t2) {
        const int p = it / nchunks;
        const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
        t1 = cand ? cand[(size_t)p * kc + j1] : j1;
        t2 = cand ? cand[(size_t)p * kc + j2] : j2;
    };
    // L2 prefetch of the template pair that follows (item, pi): the next pair of
    // the item, else the first pair (and the pattern) of this cluster's next item
    auto prefetch_next = [&](int it, int pi, int pe) {
        if (tid != 0) return;
        int nit = it, npi = pi + 1;
        if (npi >= pe) {
            nit = it + ncl;
            if (nit >= n_items || degen[nit / nchunks]) return;
            npi = (nit - (nit / nchunks) * nchunks) * ppc;
            if (npi >= npairs) return;
            prefetch_quarter(Sp + (size_t)(nit / nchunks) * N * HW, c);
        }
        int t1, t2;
        pair_templates(nit, npi, t1, t2);
        if (t1 >= 0) prefetch_packed(St + (size_t)t1 * PK_F2, c);
        if (t2 >= 0 && t2 != t1) prefetch_packed(St + (size_t)t2 * PK_F2, c);
    };
    if (cid < n_items && !degen[cid / nchunks]) {   // the first pair of the first item
        const int pb0 = (cid - (cid / nchunks) * nchunks) * ppc;
        if (pb0 < npairs) {
            if (tid == 0) prefetch_quarter(Sp + (size_t)(cid / nchunks) * N * HW, c);
            prefetch_next(cid, pb0 - 1, pb0 + 1);
        }
    }

    for (int item = cid; item < n_items; item += ncl) {
        const int p = item / nchunks, ch = item - p * nchunks;
        const int pb = ch * ppc, pe = min(npairs, pb + ppc);
        if (degen[p]) continue;   // uniform over the cluster
        const float2 *sp = Sp + (size_t)p * N * HW;
        unsigned long long kbest = 0;
        for (int pi = pb; pi < pe; ++pi) {
            const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
            int t1, t2;
            pair_templates(item, pi, t1, t2);
            prefetch_next(item, pi, pe);
            const float2 *s1 = St + (size_t)max(t1, 0) * PK_F2, *s2 = St + (size_t)max(t2, 0) * PK_F2;
            // ---- rows ua and ub of Z = X1 + i X2, transformed along v
            {
                float2 a[16], b[16];
                build_half<true>(s1, s2, sp, ua, l, a, b);
                build_half<true>(s1, s2, sp, singles ? ua : ub, sg, b, a);   // singles: row 0 as the pair (0, 0)
                ifft256_pass1(a, [&](int k1) { return twa[k1 * 16 + l]; }, l, scr, l);
                dif16<0, 4, +1>(a);
                if (pending) {   // every CTA is done reading this CTA's Zc
                    cluster_wait();
                    pending = false;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) Zc[zc_at(sa, l + 16 * cx_bitrev(q, 4))] = a[q];
                if (singles) {   // row 128 as the pair (128, 128), held at columns l + 16 m
                    build_half<true>(s1, s2, sp, ub, l, b, a);
                    build_half<true>(s1, s2, sp, ub, sg, a, b);
                }
                // the second row's twiddle e^{+2 pi i (16 - l) k1 / 256} = W16^k1 conj(e^{+2 pi i l k1 / 256})
                // (the singles' row 128 sits at columns l + 16 m: the plain twiddle)
                ifft256_pass1(
                    b,
                    [&](int k1) {
                        const float2 w = twa[k1 * 16 + l];
                        const float2 c = singles ? make_float2(1.f, 0.f) : make_float2(kW16c[k1], kW16s[k1]);
                        return c_mul(c, make_float2(w.x, singles ? w.y : -w.y));
                    },
                    singles ? l : ng, scr, l);
                dif16<0, 4, +1>(b);
#pragma unroll
                for (int q = 0; q < 16; ++q) Zc[zc_at(sb, l + 16 * cx_bitrev(q, 4))] = b[q];
            }
            cluster_barrier();
            // ---- columns 64 c + 2 g + q (q < 2, adjacent in every row): gather over
            // the cluster, 16 bytes per row, transform, maxima
            float m1 = -INFINITY, m2 = -INFINITY;
            {
                float2 a[16], b[16];
                StaticFor<0, 16>::run([&](auto nn) {
                    constexpr int n1 = decltype(nn)::value;
                    const float4 v = ld_cluster4(cbase + (uint32_t)(n1 * N * sizeof(float2)));
                    a[n1] = make_float2(v.x, v.y);
                    b[n1] = make_float2(v.z, v.w);
                });
                auto column_max = [&](float2(&x)[16]) {
                    ifft256_pass1(x, [&](int k1) { return twa[k1 * 16 + l]; }, l, scr, l);
                    dif16<0, 3, +1>(x);
                    // the last stage (span 1, no twiddle) folded into the maxima:
                    // max(a + b, a - b) = a + |b| per real component
#pragma unroll
                    for (int k = 0; k < 16; k += 2) {
                        m1 = fmaxf(m1, x[k].x + fabsf(x[k + 1].x));
                        m2 = fmaxf(m2, x[k].y + fabsf(x[k + 1].y));
                    }
                };
                column_max(a);
                column_max(b);
            }
            // the pattern's key is the maximum over pairs, lanes, warps and CTAs
            // of (value, lowest template): kept per lane, reduced once per item
            if (t1 >= 0) kbest = max(kbest, pack_key(m1, t1));
            if (j2 != j1 && t2 >= 0) kbest = max(kbest, pack_key(m2, t2));
            if (!peaks_all) {
                cluster_arrive_relaxed();   // completed before the next pair's first Zc store
                pending = true;
                continue;
            }
            // every surface's maximum over the cluster (correlate-all mode)
            m1 = warp_max(m1);
            m2 = warp_max(m2);
            if (lane == 0) {
                red[warp] = m1;
                red[16 + warp] = m2;
            }
            __syncthreads();
            if (tid == 0) {
                float a1 = red[0], a2 = red[16];
                for (int w = 1; w < cw::NT / 32; ++w) {
                    a1 = fmaxf(a1, red[w]);
                    a2 = fmaxf(a2, red[16 + w]);
                }
                red[32] = a1;
                red[33] = a2;
            }
            cluster_barrier();   // every column read done; red[32..33] of all CTAs final
            if (c == 0 && tid == 0) {
                float a1 = red[32], a2 = red[33];
                for (int o = 1; o < NC; ++o) {
                    const uint32_t ra = map_to_rank(red_local, o);
                    a1 = fmaxf(a1, ld_cluster_f(ra + 32 * sizeof(float)));
                    a2 = fmaxf(a2, ld_cluster_f(ra + 33 * sizeof(float)));
                }
                peaks_all[(size_t)p * n + j1] = t1 >= 0 ? a1 : -INFINITY;
                if (j2 != j1) peaks_all[(size_t)p * n + j2] = t2 >= 0 ? a2 : -INFINITY;
            }
            // red[32..33] are written again only after the next pair's row-phase
            // barrier, which CTA 0 reaches after these reads
        }
        kbest = warp_max_u64(kbest);
        if (lane == 0 && kbest) atomicMax(keys + p, kbest);
    }
    if (pending) cluster_wait();
    cluster_barrier();   // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------ single-surface peak
// Two patterns per cluster pass, one surface each (real and imaginary parts
// of one complex inverse transform): after the column phase every CTA posts
// its best (value, row-major index) per surface; CTA 0 takes the cluster's
// argmax (ties: lowest index), recomputes the three columns around each peak
// from the distributed rows and fits the parabolas (the peak up-sampling
// reading: 3 points per axis, clamped to +-0.5).
constexpr size_t PEAK_SMEM = (ZC_F2 + SCR_F2) * sizeof(float2) + (6 * N + 64) * sizeof(float);

__device__ __forceinline__ void better(float &bv, int &bi, float v, int i) {
    if (v > bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
    }
}
__device__ __forceinline__ float parabola_c(float cm, float c0, float cp) {
    const float den = cm - 2.f * c0 + cp;
    if (!(den < 0.f)) return 0.f;
    const float d = (cm - cp) / (2.f * den);
    return fminf(0.5f, fmaxf(-0.5f, d));
}

__global__ void __launch_bounds__(NT, 1)
k_pair_peak_c256(const float2 *__restrict__ St, const int *__restrict__ tidx, const float2 *__restrict__ Sp,
                 const int *__restrict__ degen, const int *__restrict__ active, int P, float *__restrict__ peak,
                 float *__restrict__ shift, int *__restrict__ argmax) {
    extern __shared__ float4 smem_raw[];
    float2 *Zc = reinterpret_cast<float2 *>(smem_raw);
    float2 *scr_all = Zc + ZC_F2;
    float *colbuf = reinterpret_cast<float *>(scr_all + SCR_F2);   // [6][256] recomputed columns
    float *cand = colbuf + 6 * N;                                   // [0..3] (value a, index a, value b, index b)
    float *wred = cand + 8;                                         // [0..31] warp candidates
    const int tid = threadIdx.x, t = tid & 15, g = tid >> 4, warp = tid >> 5, lane = tid & 31;
    const int c = (int)cluster_rank();
    const int cid = blockIdx.x / NC, ncl = gridDim.x / NC;
    float2 *scr = scr_all + g * 256;

    float2 tw[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        double sn, co;
        sincospi(2.0 * t * k / N, &sn, &co);
        tw[k] = make_float2((float)co, (float)sn);
    }
    const uint32_t zc_local = (uint32_t)__cvta_generic_to_shared(Zc);
    const uint32_t cand_local = (uint32_t)__cvta_generic_to_shared(cand);
    uint32_t rbase[16];
    int rsw[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        int owner, slot;
        row_home(16 * n1 + t, owner, slot);
        rbase[n1] = map_to_rank(zc_local, owner) + (uint32_t)(slot * N * sizeof(float2));
        rsw[n1] = (slot >> 1) & 15;
    }
    const int npass = (P + 1) / 2;
    for (int k2 = cid; k2 < npass; k2 += ncl) {
        const int pa = 2 * k2, pb = 2 * k2 + 1;
        // per surface: 0 skip (inactive / absent), 1 zero outputs, 2 compute
        int mode[2];
        int tt[2];
        for (int s = 0; s < 2; ++s) {
            const int p = s ? pb : pa;
            if (p >= P || (active && !active[p])) {
                mode[s] = 0;
                tt[s] = 0;
                continue;
            }
            tt[s] = tidx ? tidx[p] : p;
            mode[s] = ((degen && degen[p]) || tt[s] < 0) ? 1 : 2;
        }
        if (tid == 0 && c == 0)
            for (int s = 0; s < 2; ++s)
                if (mode[s] == 1) {
                    const int p = s ? pb : pa;
                    peak[p] = 0.f;
                    shift[2 * p] = 0.f;
                    shift[2 * p + 1] = 0.f;
                }
        if (mode[0] != 2 && mode[1] != 2) continue;    // uniform over the cluster
        const float2 *sa = St + (size_t)(mode[0] == 2 ? tt[0] : 0) * N * HW;
        const float2 *sb = St + (size_t)(mode[1] == 2 ? tt[1] : 0) * N * HW;
        const float2 *qa = Sp + (size_t)(mode[0] == 2 ? pa : 0) * N * HW;
        const float2 *qb = Sp + (size_t)(mode[1] == 2 ? pb : 0) * N * HW;
        rows_phase(Zc, sa, qa, mode[0] == 2 ? 1.f : 0.f, sb, qb, mode[1] == 2 ? 1.f : 0.f, tw, scr, c, g, t);
        cluster_barrier();
        float bva = -INFINITY, bvb = -INFINITY;
        int bia = 0x7fffffff, bib = 0x7fffffff;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int x = ROWS * c + 4 * g + q;
            float2 a[16];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1)
                a[n1] = ld_cluster(rbase[n1] + (uint32_t)((x ^ rsw[n1]) * sizeof(float2)));
            line_ifft(a, tw, scr, t);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int i = (t + 16 * cx_bitrev(k, 4)) * N + x;
                better(bva, bia, a[k].x, i);
                better(bvb, bib, a[k].y, i);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            better(bva, bia, __shfl_xor_sync(0xffffffffu, bva, o), __shfl_xor_sync(0xffffffffu, bia, o));
            better(bvb, bib, __shfl_xor_sync(0xffffffffu, bvb, o), __shfl_xor_sync(0xffffffffu, bib, o));
        }
        if (lane == 0) {
            wred[4 * warp] = bva;
            wred[4 * warp + 1] = __int_as_float(bia);
            wred[4 * warp + 2] = bvb;
            wred[4 * warp + 3] = __int_as_float(bib);
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < NT / 32; ++w) {
                better(bva, bia, wred[4 * w], __float_as_int(wred[4 * w + 1]));
                better(bvb, bib, wred[4 * w + 2], __float_as_int(wred[4 * w + 3]));
            }
            cand[0] = bva;
            cand[1] = __int_as_float(bia);
            cand[2] = bvb;
            cand[3] = __int_as_float(bib);
        }
        cluster_barrier();   // every CTA's candidates posted
        if (c == 0) {
            // the cluster's argmax, the same in every thread of CTA 0 (ranks in order)
            float va = -INFINITY, vb = -INFINITY;
            int ia = 0x7fffffff, ib = 0x7fffffff;
            for (int r = 0; r < NC; ++r) {
                const uint32_t ra = map_to_rank(cand_local, r);
                better(va, ia, ld_cluster_f(ra), __float_as_int(ld_cluster_f(ra + 4)));
                better(vb, ib, ld_cluster_f(ra + 8), __float_as_int(ld_cluster_f(ra + 12)));
            }
            // groups 0..5 recompute the columns x0 - 1, x0, x0 + 1 of each surface
            if (g < 6) {
                const int s = g / 3, d = g % 3 - 1;
                const int i0 = s ? ib : ia;
                const int x = ((i0 & (N - 1)) + d + N) & (N - 1);
                float2 a[16];
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1)
                    a[n1] = ld_cluster(rbase[n1] + (uint32_t)((x ^ rsw[n1]) * sizeof(float2)));
                line_ifft(a, tw, scr, t);
#pragma unroll
                for (int k = 0; k < 16; ++k) colbuf[g * N + t + 16 * cx_bitrev(k, 4)] = s ? a[k].y : a[k].x;
            }
            __syncthreads();
            if (tid < 2 && mode[tid] == 2) {
                const int s = tid, i0 = s ? ib : ia, p = s ? pb : pa;
                const float *cb = colbuf + 3 * s * N;
                const int y0 = i0 >> 8, x0 = i0 & (N - 1);
                const float c0 = cb[N + y0];
                const float cxm = cb[y0], cxp = cb[2 * N + y0];
                const float cym = cb[N + ((y0 + N - 1) & (N - 1))], cyp = cb[N + ((y0 + 1) & (N - 1))];
                peak[p] = c0;
                shift[2 * p] = (float)(x0 < N / 2 ? x0 : x0 - N) + parabola_c(cxm, c0, cxp);
                shift[2 * p + 1] = (float)(y0 < N / 2 ? y0 : y0 - N) + parabola_c(cym, c0, cyp);
                if (argmax) argmax[p] = i0;
            }
        }
        cluster_barrier();   // CTA 0 done reading the distributed rows and candidates
    }
    cluster_barrier();
}

// ------------------------------------------------------ pre-processing
// One cluster per image (Eq. 4 and the filtering / normalisation of the FFT
// section): CTA c loads rows 64c..64c+63 of the crop, the cluster reduces the
// mean and standard deviation, the rows are windowed and transformed two at a
// time (one complex line, split by Hermitian symmetry) into R[y][0..128], and
// CTA c then gathers and transforms columns 32c..32c+31 (CTA 3 also column
// 128), filters them and reduces the filtered energy over the cluster.  With a
// spatial output the filtered, normalised spectrum is transformed back:
// columns in place, then rows two at a time (conjugate-symmetric extension).
constexpr size_t RC_F2 = (size_t)ROWS * HW;                        // row spectra [64][129]
constexpr size_t ST_F2 = (size_t)N * 32;                          // column staging [256][32]
constexpr size_t IN_F = (size_t)ROWS * N;                          // input rows [64][256] of the next image
constexpr size_t PREP_SMEM = (RC_F2 + ST_F2 + N + SCR_F2) * sizeof(float2) + 16 * sizeof(double) + IN_F * sizeof(float);
static_assert(PREP_SMEM <= 232448, "pre-processing shared memory above the per-CTA limit");

__device__ __forceinline__ void cp_async_4(uint32_t s, const float *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_16(uint32_t s, const float *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(g) : "memory");
}

__device__ __forceinline__ double ld_cluster_d(uint32_t addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
// FP32 partial per thread: warp sums in FP32, the warps' sums in FP64
__device__ __forceinline__ double block_sum_fd(float v, double *sh) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}
// sum of one partial per CTA, identical (same order) in every CTA of the cluster
__device__ __forceinline__ double cluster_sum(double part, double *slot, uint32_t slot_addr) {
    if (threadIdx.x == 0) *slot = part;
    cluster_barrier();
    double s = 0.0;
    for (int r = 0; r < NC; ++r) s += ld_cluster_d(map_to_rank(slot_addr, r));
    return s;
}
__device__ __forceinline__ int st_index(int u, int vl) { return u * 32 + (vl ^ (u & 31)); }


__global__ void __launch_bounds__(NT, 1)
k_prep_c256(const float *__restrict__ img, int P, PrepArgs a, float2 *__restrict__ spec, float *__restrict__ spatial,
            int *__restrict__ degen, const int *__restrict__ active) {
    extern __shared__ float4 smem_raw[];
    float2 *Rc = reinterpret_cast<float2 *>(smem_raw);
    float2 *Stage = Rc + RC_F2;
    float2 *Col128 = Stage + ST_F2;
    float2 *scr_all = Col128 + N;
    double *red = reinterpret_cast<double *>(scr_all + SCR_F2);   // [0..7] block partials, [8..10] cluster slots
    float *Xr = reinterpret_cast<float *>(red + 16);              // this CTA's 64 input rows [64][256]
    const int tid = threadIdx.x, t = tid & 15, g = tid >> 4;
    const int c = (int)cluster_rank();
    const int cid = blockIdx.x / NC, ncl = gridDim.x / NC;
    float2 *scr = scr_all + g * 256;

    float2 tw[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        double sn, co;
        sincospi(2.0 * t * k / N, &sn, &co);
        tw[k] = make_float2((float)co, (float)sn);
    }
    const uint32_t rc_local = (uint32_t)__cvta_generic_to_shared(Rc);
    const uint32_t st_local = (uint32_t)__cvta_generic_to_shared(Stage);
    const uint32_t c128_local = (uint32_t)__cvta_generic_to_shared(Col128);
    const uint32_t slot_local = (uint32_t)__cvta_generic_to_shared(red + 8);
    uint32_t rrow[16];   // column phase: cluster address of row y = 16 n1 + t of R
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        const int y = 16 * n1 + t;
        rrow[n1] = map_to_rank(rc_local, y >> 6) + (uint32_t)((y & 63) * HW * sizeof(float2));
    }
    const float inv_nn = 1.f / N;
    // this CTA's 64 crop rows of an image into Xr, asynchronously (16-byte
    // copies when the crop's rows start on 16-byte boundaries)
    const bool v16 = ((reinterpret_cast<uintptr_t>(img) | ((uintptr_t)a.W * 4) | ((uintptr_t)a.ox * 4)) & 15) == 0;
    const uint32_t xr_local = (uint32_t)__cvta_generic_to_shared(Xr);
    auto load_rows = [&](int q) {
        const float *src = img + (size_t)q * a.W * a.H + (size_t)(a.oy + ROWS * c) * a.W + a.ox;
        if (v16) {
            for (int i = tid; i < ROWS * N / 4; i += NT)
                cp_async_16(xr_local + (uint32_t)(16 * i), src + (size_t)(i >> 6) * a.W + 4 * (i & 63));
        } else {
            for (int i = tid; i < ROWS * N; i += NT)
                cp_async_4(xr_local + (uint32_t)(4 * i), src + (size_t)(i >> 8) * a.W + (i & (N - 1)));
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto next_active = [&](int q) {   // uniform over the cluster
        while (q < P && active && !active[q]) q += ncl;
        return q;
    };
    int p = next_active(cid), pn = P;
    if (p < P) load_rows(p);

    for (; p < P; p = pn) {
        pn = next_active(p + ncl);
        const float *src = img + (size_t)p * a.W * a.H;
        float2 *out = spec + (size_t)p * N * HW;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();   // Xr holds image p
        // ---- statistics of the crop: one pass of FP32 sums of (x - x0), x0 the crop's
        // first pixel (the same in every CTA; a constant crop has exactly zero variance),
        // combined in FP64, one cluster barrier for both
        const float x0 = __ldg(src + (size_t)a.oy * a.W + a.ox);
        float sf = 0.f, sf2 = 0.f;
        for (int i = tid; i < ROWS * N; i += NT) {
            const float v = Xr[i];
            const float d = v - x0;
            sf += d;
            sf2 = fmaf(d, d, sf2);
        }
        const double s = block_sum_fd(sf, red);
        const double s2 = block_sum_fd(sf2, red);
        if (tid == 0) red[9] = s2;
        const double tot = cluster_sum(s, red + 8, slot_local);   // its barrier also publishes red[9]
        double tot2 = 0.0;
        for (int r = 0; r < NC; ++r) tot2 += ld_cluster_d(map_to_rank(slot_local + sizeof(double), r));
        const double m1 = tot / ((double)N * N);
        const double mean = x0 + m1;
        const double sd = sqrt(fmax(tot2 / ((double)N * N) - m1 * m1, 0.0));
        bool bad = !(sd > 1e-12 * (1.0 + fabs(mean)));
        if (!bad) {
            // ---- rows (two per complex line), windowed and standardised
            const float m = (float)mean, inv = (float)(1.0 / sd);
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                const int ra = 2 * (g + 16 * q), rb = ra + 1;
                const int ya = ROWS * c + ra, yb = ya + 1;
                const float wa = a.window ? 0.5f * (1.f - cospif(2.f * ya / N)) : 1.f;
                const float wb = a.window ? 0.5f * (1.f - cospif(2.f * yb / N)) : 1.f;
                float2 z[16];
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) {
                    const int x = 16 * n1 + t;
                    // cos(2 pi x / 256) = Re(W16^n1 e^{2 pi i t / 256}), the latter in tw[1]
                    const float cx = kW16c[n1] * tw[1].x - kW16s[n1] * tw[1].y;
                    const float wx = (a.window ? 0.5f * (1.f - cx) : 1.f) * inv;
                    z[n1] = make_float2((Xr[ra * N + x] - m) * wx * wa, (Xr[rb * N + x] - m) * wx * wb);
                }
                line_fft<-1>(z, tw, scr, t);
#pragma unroll
                for (int k = 0; k < 16; ++k) scr[t + 16 * cx_bitrev(k, 4)] = z[k];
                __syncwarp(0xffffu << (tid & 16));
#pragma unroll
                for (int mm = 0; mm < 9; ++mm) {
                    const int v = t + 16 * mm;
                    if (v > 128) break;
                    const float2 zv = scr[v], zn = scr[(N - v) & (N - 1)];
                    Rc[ra * HW + v] = make_float2(0.5f * (zv.x + zn.x), 0.5f * (zv.y - zn.y));
                    Rc[rb * HW + v] = make_float2(0.5f * (zv.y + zn.y), 0.5f * (zn.x - zv.x));
                }
                __syncwarp(0xffffu << (tid & 16));
            }
        }
        cluster_barrier();   // R complete (every CTA takes the same branch: mean and sd are cluster-wide)
        if (pn < P) load_rows(pn);   // every warp of this CTA is done with Xr
        float e = 0.f;
        if (!bad) {
            // ---- columns: gather, transform, filter; keep in Stage / Col128
            const int nq = (c == NC - 1 && g == 0) ? 3 : 2;
            // the band-pass as per-frequency factors, e = expm1(-f^2 / 2 s_h^2),
            // b = exp(-f^2 / 2 s_l^2): h = -(e_u + e_v + e_u e_v) b_u b_v; the
            // lane's 16 row factors once per image
            float eu[16], bu[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int u = t + 16 * cx_bitrev(k, 4);
                const float fu = (float)(u < N / 2 ? u : u - N), f2 = fu * fu;
                eu[k] = expm1f(-f2 * a.inv2shp);
                bu[k] = expf(-f2 * a.inv2slp);
            }
#pragma unroll 1
            for (int q = 0; q < nq; ++q) {
                const int v = q < 2 ? 32 * c + 2 * g + q : 128;
                float2 z[16];
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) z[n1] = ld_cluster(rrow[n1] + (uint32_t)(v * sizeof(float2)));
                line_fft<-1>(z, tw, scr, t);
                const float fv = (float)(v < N / 2 ? v : v - N), fv2 = fv * fv;
                const float ev = expm1f(-fv2 * a.inv2shp), bv = expf(-fv2 * a.inv2slp);
                const float wv = (v == 0 || v == N / 2) ? 1.f : 2.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int u = t + 16 * cx_bitrev(k, 4);
                    const float h = -(eu[k] + ev + eu[k] * ev) * (bu[k] * bv);
                    const float2 X = make_float2(z[k].x * h, z[k].y * h);
                    e = fmaf(wv, X.x * X.x + X.y * X.y, e);
                    if (q < 2) Stage[st_index(u, v - 32 * c)] = X;
                    else Col128[u] = X;
                }
            }
        }
        const double energy = cluster_sum(block_sum_fd(e, red), red + 10, slot_local + 2 * sizeof(double));
        bad = bad || !(energy > 0.0);
        if (tid == 0 && c == 0 && degen) degen[p] = bad ? 1 : 0;
        if (bad) {
            for (int i = tid; i < ROWS * HW; i += NT) out[(size_t)ROWS * c * HW + i] = make_float2(0.f, 0.f);
            if (spatial)
                for (int i = tid; i < ROWS * N; i += NT) spatial[(size_t)p * N * N + (size_t)ROWS * c * N + i] = 0.f;
            continue;   // uniform: the decision used cluster-wide sums
        }
        const float sc = (float)(1.0 / sqrt(energy));
        for (int i = tid; i < N * 32; i += NT) {
            const int u = i >> 5, vl = i & 31;
            const float2 X = Stage[st_index(u, vl)];
            out[(size_t)u * HW + 32 * c + vl] = make_float2(X.x * sc, X.y * sc);
        }
        if (c == NC - 1)
            for (int u = tid; u < N; u += NT) out[(size_t)u * HW + 128] = make_float2(Col128[u].x * sc, Col128[u].y * sc);
        if (!spatial) continue;   // Stage is written again after the next image's row barrier
        __syncthreads();
        // ---- spatial image: columns back in place, then rows two at a time
        {
            const int nq = (c == NC - 1 && g == 0) ? 3 : 2;
#pragma unroll 1
            for (int q = 0; q < nq; ++q) {
                const int vl = 2 * g + q;
                float2 z[16];
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) {
                    const int u = 16 * n1 + t;
                    const float2 X = q < 2 ? Stage[st_index(u, vl)] : Col128[u];
                    z[n1] = make_float2(X.x * sc, X.y * sc);
                }
                line_fft<+1>(z, tw, scr, t);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int y = t + 16 * cx_bitrev(k, 4);
                    if (q < 2) Stage[st_index(y, vl)] = z[k];
                    else Col128[y] = z[k];
                }
            }
        }
        cluster_barrier();   // T[y][v] of every column visible
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            const int ya = ROWS * c + 2 * (g + 16 * q), yb = ya + 1;
            float2 z[16];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                const int v = 16 * n1 + t;
                const int w = v <= 128 ? v : N - v;
                float2 ta, tb;
                if (w == 128) {
                    const uint32_t base = map_to_rank(c128_local, NC - 1);
                    ta = ld_cluster(base + (uint32_t)(ya * sizeof(float2)));
                    tb = ld_cluster(base + (uint32_t)(yb * sizeof(float2)));
                } else {
                    const uint32_t base = map_to_rank(st_local, w >> 5);
                    ta = ld_cluster(base + (uint32_t)(st_index(ya, w & 31) * sizeof(float2)));
                    tb = ld_cluster(base + (uint32_t)(st_index(yb, w & 31) * sizeof(float2)));
                }
                if (v > 128) {   // conjugate-symmetric extension of a real image's row
                    ta.y = -ta.y;
                    tb.y = -tb.y;
                }
                z[n1] = make_float2(ta.x - tb.y, ta.y + tb.x);
            }
            line_fft<+1>(z, tw, scr, t);
            float *oa = spatial + (size_t)p * N * N + (size_t)ya * N, *ob = oa + N;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int x = t + 16 * cx_bitrev(k, 4);
                oa[x] = z[k].x * inv_nn;
                ob[x] = z[k].y * inv_nn;
            }
        }
        cluster_barrier();   // Stage / Col128 read by the other CTAs: free for the next image
    }
    cluster_barrier();
}

template <class K>
int max_active_clusters(K kernel, int nt, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(NC * 64);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 32;
    }
    return n;
}

}  // namespace

size_t c256_search_layout_f2() { return cw::PK_F2; }

cudaError_t launch_pack_c256(const float2 *spectra, int T, float2 *packed, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    const size_t total = (size_t)T * cw::PK_F2;
    const int blocks = (int)((total + 255) / 256 < 65536 ? (total + 255) / 256 : 65536);
    cw::k_pack_c256<<<blocks, 256, 0, st>>>(spectra, T, packed);
    return cudaGetLastError();
}

cudaError_t launch_search_c256(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                               unsigned long long *keys, float *peaks_all, const int *cand, int kc,
                               cudaStream_t st) {
    const int n = cand ? kc : T;
    if (P <= 0 || n <= 0) return cudaSuccess;
    auto *kernel = k_search_c256w;
    const int nt = cw::NT;
    const size_t smem = cw::SMEM_BYTES;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int npairs = (n + 1) / 2;
    static const int ncl_max = max_active_clusters(kernel, nt, smem);
    // chunks of pairs so that there are at least ~4 items per resident cluster
    const long want = 4L * ncl_max;
    int nchunks = (int)((want + P - 1) / P);
    nchunks = nchunks < 1 ? 1 : (nchunks > npairs ? npairs : nchunks);
    const int ppc = (npairs + nchunks - 1) / nchunks;
    nchunks = (npairs + ppc - 1) / ppc;
    const long n_items = (long)P * nchunks;
    if (n_items > (1L << 30)) return cudaErrorInvalidValue;
    const int ncl = (int)(n_items < ncl_max ? n_items : ncl_max);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(NC * ncl);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, St, T, Sp, degen, nchunks, ppc, (int)n_items, keys, peaks_all, cand, kc);
}

cudaError_t launch_prep_c256(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                             const int *active, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (a.N != N) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_prep_c256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PREP_SMEM);
    if (e != cudaSuccess) return e;
    static int ncl_max = -1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = PREP_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ncl_max < 0) {
        cfg.gridDim = dim3(NC * 64);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_prep_c256, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 32;
        }
        ncl_max = n;
    }
    const int ncl = P < ncl_max ? P : ncl_max;
    cfg.gridDim = dim3(NC * ncl);
    return cudaLaunchKernelEx(&cfg, k_prep_c256, img, P, a, spec, spatial, degen, active);
}

cudaError_t launch_pair_peak_c256(const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                  const int *active, int P, float *peak, float *shift, cudaStream_t st,
                                  int *argmax) {
    if (P <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_pair_peak_c256, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PEAK_SMEM);
    if (e != cudaSuccess) return e;
    static int ncl_max = -1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = PEAK_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ncl_max < 0) {
        cfg.gridDim = dim3(NC * 64);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_pair_peak_c256, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 32;
        }
        ncl_max = n;
    }
    const int npass = (P + 1) / 2;
    const int ncl = npass < ncl_max ? npass : ncl_max;
    cfg.gridDim = dim3(NC * ncl);
    return cudaLaunchKernelEx(&cfg, k_pair_peak_c256, St, tidx, Sp, degen, active, P, peak, shift, argmax);
}
