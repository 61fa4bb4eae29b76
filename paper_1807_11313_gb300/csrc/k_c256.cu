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
constexpr size_t SMEM_BYTES = (ZC_F2 + SCR_F2) * sizeof(float2) + 64 * sizeof(float);

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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
__device__ __forceinline__ float ld_cluster_f(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

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

// 256-point inverse DFT (X[k] = sum_n x[n] e^{+2 pi i nk/256}) of a line held
// by a 16-thread group: on entry a[n1] = x[16 n1 + t]; on exit a[p] =
// X[t + 16 bitrev4(p)].  tw[k] = e^{+2 pi i t k / 256}; scr = the group's buffer.
__device__ __forceinline__ void line_ifft(float2 (&a)[16], const float2 (&tw)[16], float2 *scr, int t) {
    fft_reg_dif<16, +1>(a);   // a[p] = A[bitrev(p)], A[k1] = sum_n1 x[16 n1 + t] e^{+2 pi i n1 k1 / 16}
    StaticFor<0, 16>::run([&](auto pp) {
        constexpr int p = decltype(pp)::value;
        constexpr int k1 = cx_bitrev(p, 4);
        const float2 v = k1 == 0 ? a[p] : c_mul(a[p], tw[k1]);
        scr[t * 16 + (k1 ^ t)] = v;
    });
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) a[n2] = scr[n2 * 16 + (t ^ n2)];
    __syncwarp();
    fft_reg_dif<16, +1>(a);   // a[p] = X[t + 16 bitrev(p)]
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// pattern p, template pairs [pb, pe) (slot indices into cand when cand != null)
__global__ void __launch_bounds__(NT, 1)
k_search_c256(const float2 *__restrict__ St, int T, const float2 *__restrict__ Sp, const int *__restrict__ degen,
              int nchunks, int ppc, int n_items, unsigned long long *__restrict__ keys, float *__restrict__ peaks_all,
              const int *__restrict__ cand, int kc) {
    extern __shared__ float4 smem_raw[];
    float2 *Zc = reinterpret_cast<float2 *>(smem_raw);
    float2 *scr_all = Zc + ZC_F2;
    float *red = reinterpret_cast<float *>(scr_all + SCR_F2);   // [0..15] warp maxima, [32..33] CTA maxima
    const int tid = threadIdx.x, t = tid & 15, g = tid >> 4, warp = tid >> 5, lane = tid & 31;
    const int c = (int)cluster_rank();
    const int cid = blockIdx.x / NC, ncl = gridDim.x / NC;
    float2 *scr = scr_all + g * 256;
    const int n = cand ? kc : T;
    const int npairs = (n + 1) / 2;

    float2 tw[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        double s, co;
        sincospi(2.0 * t * k / N, &s, &co);
        tw[k] = make_float2((float)co, (float)s);
    }
    // column phase: cluster address of row u = 16 n1 + t in its owner's buffer
    const uint32_t zc_local = (uint32_t)__cvta_generic_to_shared(Zc);
    uint32_t rbase[16];
    int rsw[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        int owner, slot;
        row_home(16 * n1 + t, owner, slot);
        rbase[n1] = map_to_rank(zc_local, owner) + (uint32_t)(slot * N * sizeof(float2));
        rsw[n1] = (slot >> 1) & 15;
    }
    const uint32_t red_local = (uint32_t)__cvta_generic_to_shared(red);

    for (int item = cid; item < n_items; item += ncl) {
        const int p = item / nchunks, ch = item - p * nchunks;
        const int pb = ch * ppc, pe = min(npairs, pb + ppc);
        if (degen[p]) continue;                       // uniform over the cluster
        const float2 *sp = Sp + (size_t)p * N * HW;
        float best_v = -INFINITY;
        int best_t = -1;
        for (int pi = pb; pi < pe; ++pi) {
            const int j1 = 2 * pi, j2 = min(j1 + 1, n - 1);
            const int t1 = cand ? cand[(size_t)p * kc + j1] : j1;
            const int t2 = cand ? cand[(size_t)p * kc + j2] : j2;
            const float2 *s1 = St + (size_t)max(t1, 0) * N * HW, *s2 = St + (size_t)max(t2, 0) * N * HW;
            // ---- rows: group g builds and transforms the pairs j = g and g + 16
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
                    if (v <= 128) {
                        const int k = u * HW + v;
                        const float2 s = __ldg(sp + k);
                        const float2 x1 = c_mulcj(__ldg(s1 + k), s), x2 = c_mulcj(__ldg(s2 + k), s);
                        a[n1] = make_float2(x1.x - x2.y, x1.y + x2.x);
                    } else {   // Hermitian half: X(u, v) = conj(X(-u, 256 - v))
                        const int k = pu * HW + (N - v);
                        const float2 s = __ldg(sp + k);
                        const float2 x1 = c_mulcj(__ldg(s1 + k), s), x2 = c_mulcj(__ldg(s2 + k), s);
                        a[n1] = make_float2(x1.x + x2.y, -x1.y + x2.x);
                    }
                }
                line_ifft(a, tw, scr, t);
                const int slot = 2 * j + (r & 1);
#pragma unroll
                for (int q = 0; q < 16; ++q) Zc[zc_index(slot, t + 16 * cx_bitrev(q, 4))] = a[q];
            }
            cluster_barrier();
            // ---- columns x = 64 c + 4 g + q: gather over the cluster, transform, maxima
            float m1 = -INFINITY, m2 = -INFINITY;
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
                    m1 = fmaxf(m1, a[k].x);
                    m2 = fmaxf(m2, a[k].y);
                }
            }
            m1 = warp_max(m1);
            m2 = warp_max(m2);
            if (lane == 0) {
                red[warp] = m1;
                red[16 + warp] = m2;
            }
            __syncthreads();
            if (tid == 0) {
                float a1 = red[0], a2 = red[16];
                for (int w = 1; w < NT / 32; ++w) {
                    a1 = fmaxf(a1, red[w]);
                    a2 = fmaxf(a2, red[16 + w]);
                }
                red[32] = a1;
                red[33] = a2;
            }
            __syncthreads();
            m1 = red[32];
            m2 = red[33];
            // per-CTA partial maxima: the key of the pattern is the max over CTAs
            if (t1 >= 0 && (m1 > best_v || (m1 == best_v && t1 < best_t))) { best_v = m1; best_t = t1; }
            if (j2 != j1 && t2 >= 0 && (m2 > best_v || (m2 == best_v && t2 < best_t))) { best_v = m2; best_t = t2; }
            cluster_barrier();                        // every column read done; red[32..33] of all CTAs final
            if (peaks_all && c == 0 && tid == 0) {   // the surfaces' maxima over the four CTAs
                float a1 = m1, a2 = m2;
                for (int o = 1; o < NC; ++o) {
                    const uint32_t ra = map_to_rank(red_local, o);
                    a1 = fmaxf(a1, ld_cluster_f(ra + 32 * sizeof(float)));
                    a2 = fmaxf(a2, ld_cluster_f(ra + 33 * sizeof(float)));
                }
                peaks_all[(size_t)p * n + j1] = t1 >= 0 ? a1 : -INFINITY;
                if (j2 != j1) peaks_all[(size_t)p * n + j2] = t2 >= 0 ? a2 : -INFINITY;
            }
        }
        if (tid == 0 && best_t >= 0) atomicMax(keys + p, pack_key(best_v, best_t));
    }
    cluster_barrier();   // no CTA leaves while another may still read its shared memory
}

int max_active_clusters() {
    static int cached = -1;
    if (cached >= 0) return cached;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(NC * 64);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_search_c256, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 32;
    }
    cached = n;
    return n;
}

}  // namespace

size_t c256_smem_bytes() { return SMEM_BYTES; }

cudaError_t launch_search_c256(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                               unsigned long long *keys, float *peaks_all, const int *cand, int kc,
                               cudaStream_t st) {
    const int n = cand ? kc : T;
    if (P <= 0 || n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_search_c256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int npairs = (n + 1) / 2;
    const int ncl_max = max_active_clusters();
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
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_search_c256, St, T, Sp, degen, nchunks, ppc, (int)n_items, keys, peaks_all,
                              cand, kc);
}
