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
// (templates) tile of S.  Warp 0 is the loader: one thread issues TMA
// (cp.async.bulk.tensor) copies of 64-wide K-slices of both operands into a
// four-stage ring, 128-byte swizzled, each stage completing an mbarrier by
// transaction count.  Warp 1 is the tensor-core issuer: one thread waits for
// a stage, issues four tcgen05.mma (M = 128, N = 256, K = 16, BF16 in, FP32
// accumulated in 256 TMEM columns) and commits them to the stage's "empty"
// mbarrier, which hands the stage back to the loader.  After the last commit
// all four warps read the accumulator with tcgen05.ld (each warp its 32 TMEM
// lanes = tile rows) and write S.  Tiles are ordered in groups of eight
// pattern tiles, so that the CTAs resident at one time share the template
// tiles they stream.  Every wait is bounded: on time-out the kernel records an
// error flag, waits (bounded) for its copies in flight and frees its tensor
// memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4, NT = 128, GROUP_M = 8;
constexpr int A_BYTES = BM * BK * 2;              // 16 KB
constexpr int B_BYTES = BN * BK * 2;              // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 48 KB
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 128;
constexpr unsigned kSpinLimit = 1u << 26;         // bounded waits

// shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzling: start address, leading byte offset 16 (unused for
// this layout), stride byte offset 1024 (between 8-row groups), version 1,
// swizzle mode 2 = 128 B.  Stage bases are 1024-byte aligned, so advancing
// the start by 32 bytes per K = 16 step keeps the swizzle phase.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major,
// N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

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
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// 2-D tiled TMA load: box at (x = K element, y = row), completes `bar` by transaction bytes
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(NT, 1)
k_screen_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int P, int T, int K,
            float *__restrict__ S, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t sbase0 = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t sbase = (sbase0 + 1023u) & ~1023u;            // 1024-aligned stages (swizzle atoms)
    const uint32_t full_bar = sbase + STAGES * STAGE_BYTES;       // STAGES mbarriers: stage loaded
    const uint32_t empty_bar = full_bar + 8 * STAGES;             // STAGES mbarriers: stage consumed
    const uint32_t done_bar = empty_bar + 8 * STAGES;             // accumulator complete
    const uint32_t tmem_slot = done_bar + 8;                      // tcgen05.alloc writes here
    unsigned char *gen_base = smem_raw + (sbase - sbase0);
    volatile uint32_t *tmem_slot_ptr =
        reinterpret_cast<volatile uint32_t *>(gen_base + STAGES * STAGE_BYTES + 16 * STAGES + 8);
    volatile int *flag = reinterpret_cast<volatile int *>(gen_base + STAGES * STAGE_BYTES + 16 * STAGES + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // grouped tile order: GROUP_M pattern tiles per template-tile sweep
    const int num_m = (P + BM - 1) / BM, num_n = (T + BN - 1) / BN;
    const int id = blockIdx.x, per_group = GROUP_M * num_n;
    const int first_m = (id / per_group) * GROUP_M;
    const int gsize = min(num_m - first_m, GROUP_M);
    const int m_tile = first_m + (id % per_group) % gsize, n_tile = (id % per_group) / gsize;
    const int p0 = m_tile * BM, t0 = n_tile * BN;
    const int nk = K / BK;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full_bar + 8 * s));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty_bar + 8 * s));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done_bar));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot), "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot_ptr;

    int issued = 0;   // loader: stages issued (for the drain on a time-out)
    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(empty_bar + 8 * s, (uint32_t)((kb / STAGES - 1) & 1))) {
                *flag = 1;
                break;
            }
            if (*flag) break;
            const uint32_t sa = sbase + s * STAGE_BYTES, sb = sa + A_BYTES;
            mbar_expect_tx(full_bar + 8 * s, STAGE_BYTES);
            tma_load_2d(sa, &mapA, kb * BK, p0, full_bar + 8 * s);
            tma_load_2d(sb, &mapB, kb * BK, t0, full_bar + 8 * s);
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0) {
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(full_bar + 8 * s, (uint32_t)((kb / STAGES) & 1)) || *flag) {
                *flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = sbase + s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = smem_desc_sw128(sa + kk * 32), bd = smem_desc_sw128(sb + kk * 32);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                empty_bar + 8 * s));
        }
        // the done barrier fires when every MMA issued above has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done_bar));
    }
    __syncwarp();
    bool ok = mbar_wait(done_bar, 0u);
    if (!ok) *flag = 1;
    __syncthreads();
    const bool good = *flag == 0;
    if (!good && warp == 0 && lane == 0) {
        // drain: every issued stage's copies must land before the shared memory is released
        for (int kb = 0; kb < issued; ++kb) {
            const int s = kb % STAGES;
            if (kb + STAGES >= issued) mbar_wait(full_bar + 8 * s, (uint32_t)((kb / STAGES) & 1));
        }
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (good) {
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

namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}
// rows x K BF16 matrix (row-major), boxes of box_rows x 64 (128 bytes, the swizzle span)
bool make_map(CUtensorMap *m, const void *base, int rows, int K, int box_rows) {
    EncodeTiled f = encode_fn();
    if (!f) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t launch_screen_tc(const void *A, int P, const void *B, int T, int K, float *S, int *err,
                             cudaStream_t st) {
    if (P <= 0 || T <= 0) return cudaSuccess;
    // TMA: 16-byte aligned bases and row strides; K a multiple of the 64-element slice
    if (K % BK || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, P, K, BM) || !make_map(&mb, B, T, K, BN)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const long tiles = (long)((P + BM - 1) / BM) * ((T + BN - 1) / BN);
    if (tiles > 0x7fffffffL) return cudaErrorInvalidValue;
    k_screen_tc<<<(unsigned)tiles, NT, SMEM_BYTES, st>>>(ma, mb, P, T, K, S, err);
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
