// Zero-shift correlation screen on the 5th-generation tensor cores.
//
// Paper: Eq. 1 (the normalised dot product is the correlation at zero shift)
// and Eq. 3 (the FFT cross-correlation it is a special case of).  Score[p, t]
// = <y_p, y_t>, the inner product of the unit-norm filtered, windowed spatial
// images, is r(0) of the XCF surface; computed here as a GEMM
// S = Yp . Yt^T with BF16 operands and FP32 accumulation, it ranks the
// library cheaply before the FP32 FFT cross-correlation rescores the best k.
//
// k_screen_tc: one CTA (128 threads) computes a 128 (patterns) x 256
// (templates) tile of S.  K-slices of 64 are staged by cp.async into shared
// memory in the canonical no-swizzle K-major layout (8 x 16-byte core
// matrices), three stages deep; one thread issues tcgen05.mma (M = 128,
// N = 256, K = 16) with the accumulator in tensor memory and commits each
// stage to an mbarrier that releases the stage for reuse.  The epilogue reads
// the accumulator with tcgen05.ld (each warp its 32 lanes = rows) and writes
// S.  Every wait is bounded: on time-out the kernel records an error flag,
// drains its copies and frees its tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3, NT = 128;
constexpr int A_BYTES = BM * BK * 2;              // 16 KB
constexpr int B_BYTES = BN * BK * 2;              // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 48 KB
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 64;
constexpr unsigned kSpinLimit = 1u << 26;         // bounded waits

// byte offset of element (row, k) of a tile in the canonical K-major layout:
// core matrix (row / 8, k / 8) of 8 rows x 16 bytes at ((row/8) * 8 + k/8) * 128
__device__ __forceinline__ int kmajor_off(int row, int k) {
    return (((row >> 3) * (BK / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// shared-memory matrix descriptor: start address, leading byte offset (between
// core matrices adjacent in K) = 128, stride byte offset (between 8-row
// groups) = 1024, version bits 46-48 = 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major,
// N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void cp_async16_zfill(uint32_t saddr, const void *g, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N_>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N_) : "memory"); }

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (unsigned spin = 0; spin < kSpinLimit; ++spin) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(NT, 1)
k_screen_tc(const __nv_bfloat16 *__restrict__ A, int P, const __nv_bfloat16 *__restrict__ B, int T, int K,
            float *__restrict__ S, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned stage base
    const uint32_t sbase0 = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t sbase = (sbase0 + 1023u) & ~1023u;
    const uint32_t bar_base = sbase + STAGES * STAGE_BYTES;      // STAGES mbarriers (8 B each)
    const uint32_t tmem_slot = bar_base + 8 * STAGES;            // tcgen05.alloc writes here
    unsigned char *gen_base = smem_raw + (sbase - sbase0);
    volatile uint32_t *tmem_slot_ptr = reinterpret_cast<volatile uint32_t *>(gen_base + STAGES * STAGE_BYTES + 8 * STAGES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t0 = blockIdx.x * BN, p0 = blockIdx.y * BM;
    const int nk = K / BK;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_base + 8 * s));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot), "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot_ptr;

    auto load_stage = [&](int kb, int s) {
        const uint32_t sa = sbase + s * STAGE_BYTES, sb = sa + A_BYTES;
        const int k0 = kb * BK;
#pragma unroll
        for (int i = 0; i < (BM * BK / 8) / NT; ++i) {            // A: 8 chunks per thread
            const int idx = i * NT + tid, row = idx >> 3, kc = idx & 7;
            const int p = p0 + row;
            const __nv_bfloat16 *g = A + (size_t)(p < P ? p : 0) * K + k0 + kc * 8;
            cp_async16_zfill(sa + kmajor_off(row, kc * 8), g, p < P ? 16 : 0);
        }
#pragma unroll
        for (int i = 0; i < (BN * BK / 8) / NT; ++i) {            // B: 16 chunks per thread
            const int idx = i * NT + tid, row = idx >> 3, kc = idx & 7;
            const int t = t0 + row;
            const __nv_bfloat16 *g = B + (size_t)(t < T ? t : 0) * K + k0 + kc * 8;
            cp_async16_zfill(sb + kmajor_off(row, kc * 8), g, t < T ? 16 : 0);
        }
    };

    bool ok = true;
    load_stage(0, 0);
    cp_commit();
    if (nk > 1) load_stage(1, 1);
    cp_commit();
    for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        cp_wait<1>();                                             // this thread's copies of stage s landed
        asm volatile("fence.proxy.async.shared::cta;");           // visible to the tensor core
        ok = __syncthreads_and(ok ? 1 : 0) != 0;                  // block-uniform: every thread leaves together
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = sbase + s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = smem_desc(sa + kk * 256), bd = smem_desc(sb + kk * 256);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar_base + 8 * s));
        }
        // refill the stage read by the previous k-block once its MMAs are done
        if (kb + 2 < nk) {
            const int s2 = (kb + 2) % STAGES;
            if (kb >= 1) ok = mbar_wait(bar_base + 8 * s2, (uint32_t)(((kb - 1) / STAGES) & 1));
            if (ok) load_stage(kb + 2, s2);
        }
        cp_commit();
    }
    // all MMAs complete once the last k-block's commit has arrived
    if (ok) ok = mbar_wait(bar_base + 8 * ((nk - 1) % STAGES), (uint32_t)(((nk - 1) / STAGES) & 1));
    cp_wait<0>();
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int ok_all = __syncthreads_and(ok ? 1 : 0);
    if (ok_all) {
        const int row = warp * 32 + lane, p = p0 + row;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (p < P) {
                float *dst = S + (size_t)p * T + t0 + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (t0 + c0 + j < T) dst[j] = __uint_as_float(v[j]);
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// --------------------------------------------------------------------------
// top-k of each row of S (k <= 64): the k-th largest key by a 4-pass radix
// select on order-preserving 32-bit keys, then the keys above it plus the
// lowest-index keys equal to it, sorted by (score desc, index asc)
constexpr int TK_THREADS = 256;

__global__ void __launch_bounds__(TK_THREADS) k_topk_rows(const float *__restrict__ S, int P, int T, int k,
                                                          int *__restrict__ cand, float *__restrict__ score) {
    extern __shared__ uint32_t keys[];      // T keys of the row
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_need;
    __shared__ int s_count;
    __shared__ uint32_t ck[64];
    __shared__ int ci[64];
    const int p = blockIdx.x, tid = threadIdx.x;
    const float *row = S + (size_t)p * T;
    for (int i = tid; i < T; i += TK_THREADS) keys[i] = float_to_ordered(row[i]);
    if (tid == 0) { s_prefix = 0; s_need = (uint32_t)min(k, T); s_count = 0; }
    __syncthreads();
    uint32_t mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        hist[tid] = 0;
        __syncthreads();
        const uint32_t pre = s_prefix;
        for (int i = tid; i < T; i += TK_THREADS)
            if ((keys[i] & mask) == pre) atomicAdd(&hist[(keys[i] >> shift) & 255], 1u);
        __syncthreads();
        if (tid == 0) {
            uint32_t need = s_need, d = 255;
            for (;; --d) {                  // from the top digit down
                if (hist[d] >= need || d == 0) break;
                need -= hist[d];
            }
            s_prefix = pre | (d << shift);
            s_need = need;
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    const uint32_t tau = s_prefix;          // the k-th largest key
    const int kk = min(k, T);
    // keys above tau (fewer than kk), then the lowest indices equal to tau
    for (int base = 0; base < T; base += TK_THREADS) {
        const int i = base + tid;
        const bool gt = i < T && keys[i] > tau;
        if (gt) {
            const int slot = atomicAdd(&s_count, 1);
            ck[slot] = keys[i];
            ci[slot] = i;
        }
    }
    __syncthreads();
    const int ngt = s_count;
    __shared__ int s_eq_taken;
    if (tid == 0) s_eq_taken = 0;
    __syncthreads();
    for (int base = 0; base < T && s_eq_taken < kk - ngt; base += TK_THREADS) {
        const int i = base + tid;
        const bool eq = i < T && keys[i] == tau;
        // rank among equal keys of this chunk in index order (warp ballots)
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        __shared__ int wcount[TK_THREADS / 32];
        if ((tid & 31) == 0) wcount[tid >> 5] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < (tid >> 5); ++w) before += wcount[w];
        before += __popc(bal & ((1u << (tid & 31)) - 1u));
        const int taken = s_eq_taken;
        if (eq && taken + before < kk - ngt) {
            ck[ngt + taken + before] = keys[i];
            ci[ngt + taken + before] = i;
        }
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < TK_THREADS / 32; ++w) tot += wcount[w];
            s_eq_taken = min(kk - ngt, taken + tot);
        }
        __syncthreads();
    }
    // sort the kk candidates: score descending, index ascending (odd-even transposition)
    for (int pass = 0; pass < kk; ++pass) {
        const int i = 2 * tid + (pass & 1);
        if (i + 1 < kk) {
            const bool swap = ck[i] < ck[i + 1] || (ck[i] == ck[i + 1] && ci[i] > ci[i + 1]);
            if (swap) {
                const uint32_t tk = ck[i]; ck[i] = ck[i + 1]; ck[i + 1] = tk;
                const int ti = ci[i]; ci[i] = ci[i + 1]; ci[i + 1] = ti;
            }
        }
        __syncthreads();
    }
    if (tid < k) {
        cand[(size_t)p * k + tid] = tid < kk ? ci[tid] : -1;
        score[(size_t)p * k + tid] = tid < kk ? ordered_to_float(ck[tid]) : -INFINITY;
    }
}

__global__ void k_to_bf16(const float *__restrict__ x, size_t n, __nv_bfloat16 *__restrict__ y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace

cudaError_t launch_screen_tc(const void *A, int P, const void *B, int T, int K, float *S, int *err,
                             cudaStream_t st) {
    if (P <= 0 || T <= 0) return cudaSuccess;
    if (K % BK) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    dim3 grid((T + BN - 1) / BN, (P + BM - 1) / BM);
    k_screen_tc<<<grid, NT, SMEM_BYTES, st>>>(static_cast<const __nv_bfloat16 *>(A), P,
                                              static_cast<const __nv_bfloat16 *>(B), T, K, S, err);
    return cudaGetLastError();
}

cudaError_t launch_topk_rows(const float *S, int P, int T, int k, int *cand, float *score, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    if (k < 1 || k > 64) return cudaErrorInvalidValue;
    const size_t sm = sizeof(uint32_t) * (size_t)T;
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_topk_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_topk_rows<<<P, TK_THREADS, sm, st>>>(S, P, T, k, cand, score);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *x, size_t n, void *y, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = (n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536;
    k_to_bf16<<<(unsigned)blocks, 256, 0, st>>>(x, n, static_cast<__nv_bfloat16 *>(y));
    return cudaGetLastError();
}
