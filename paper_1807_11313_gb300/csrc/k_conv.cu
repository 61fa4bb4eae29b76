// 3 x 3 stride-2 convolution with bias and ReLU on the 5th-generation tensor
// cores: the BF16 inference form of the proposal network's convolutions 2-5.
//
// An implicit GEMM over NHWC activations.  Output row m = (b, oy, ox) and
// reduction index k = (ky * 3 + kx) Ci + ci give A(m, k) =
// x[b][2 oy - 1 + ky][2 ox - 1 + kx][ci] (zero outside the image: the padding
// of one pixel) and B(n, k) = w[n][ci][ky][kx], stored [Co][Kp] with Kp = 9 Ci
// rounded up to a multiple of 64 (zero columns beyond 9 Ci); y[m][n] =
// relu(bias[n] + sum_k A(m, k) B(n, k)) in FP32, stored as BF16 for the next
// layer (the rounding the next layer applies to its input anyway) or as FP32
// for the mean pool after the last layer.
//
// k_conv_tc: persistent, one CTA of 288 threads per SM, tiles of 128 output
// rows x Co channels.  Warps 0-3 are the producers: for each 64-wide K slice
// they gather the 128 A rows (16-byte cp.async, zero-filled at the image
// border and past the last row) and the weights' slice into a six-stage ring,
// both in the 128-byte swizzled K-major layout the tensor core reads (row r at
// 128 r, its 16-byte chunk c at (c ^ (r mod 8)) 16 within 1024-byte aligned
// stages).  A producer completes its copies LAG stages behind the newest,
// fences them into the async proxy and arrives on the stage's "full" barrier.
// Warp 8's first thread issues the tcgen05.mma (M = 128, N = Co, K = 16,
// BF16 in, FP32 accumulated in tensor memory, two accumulator buffers of Co
// columns) and commits each stage back to the producers through its "empty"
// barrier and each finished tile to the epilogue.  Warps 4-7 are the
// epilogue: each reads its 32 tensor-memory lanes (= tile rows) with
// tcgen05.ld, adds the bias, applies the ReLU and stores the NHWC rows while
// the next tile accumulates in the other buffer.  Every wait is bounded in
// time: on expiry the kernel raises its flag, lets its copies and products in
// flight finish, frees its tensor memory and reports through err.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {
namespace cv {

constexpr int BM = 128, BK = 64, STAGES = 6, LAG = 4;
constexpr int NPROD = 128, NEPI = 128, NT = NPROD + NEPI + 32;   // warps 0-3, 4-7, 8
constexpr int A_BYTES = BM * BK * 2;                               // 16 KB per stage
constexpr unsigned long long kWaitNs = 2000000000ull;              // 2 s per wait

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
__host__ __device__ constexpr int kp_of(int ci) { return (9 * ci + BK - 1) / BK * BK; }
__host__ __device__ constexpr size_t smem_bytes(int co) {
    return (size_t)STAGES * (A_BYTES + co * BK * 2) + 1024;   // + alignment of the ring
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: start address, leading byte offset 16 (unused for this
// layout), stride byte offset 1024 (between 8-row groups), version 1,
// swizzle mode 2 = 128 B; advancing the start by 32 bytes steps K by 16
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// wait for the phase of `parity` of `bar`: false on expiry (raising the flag)
// or, with abortable, as soon as another role has raised it
__device__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *flag, bool abortable = true) {
    if (try_wait(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (try_wait(bar, parity)) return true;
        if (abortable && *flag) return false;
        if (now_ns() - t0 > kWaitNs) {
            *flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// 16-byte copy global -> shared; n = 0 writes 16 zero bytes and reads nothing
__device__ __forceinline__ void cp16_zfill(uint32_t dst, const void *src, uint32_t n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp16_l2(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void commit_to(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace cv

// CI input channels of an S x S input, CO output channels; F32 selects an FP32 output
template <int CI, int CO, int S, bool F32>
__global__ void __launch_bounds__(cv::NT, 1)
    k_conv_tc(const __nv_bfloat16 *__restrict__ x, int B, const __nv_bfloat16 *__restrict__ w,
              const float *__restrict__ bias, void *__restrict__ y, int *__restrict__ err) {
    using namespace cv;
    constexpr int SO = S / 2, LGSO = ilog2(SO), LGCI = ilog2(CI), KP = kp_of(CI), NKB = KP / BK;
    constexpr int B_BYTES = CO * BK * 2, TM_COLS = 2 * CO;
    // kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = CO, M = 128
    constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    static_assert((1 << LGSO) == SO && (1 << LGCI) == CI && CI >= 8, "power-of-two sides and channels");
    static_assert(CO % 32 == 0 && CO >= 32 && CO <= 128, "N of the product: 32..128, a multiple of 32");
    static_assert(TM_COLS == 64 || TM_COLS == 128 || TM_COLS == 256, "tensor memory: a power of two >= 32");

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2 * STAGES + 5];
    __shared__ float bias_s[CO];
    __shared__ uint32_t tmem_slot;
    __shared__ int flag_s;
    volatile int *flag = &flag_s;

    const uint32_t abase = (smem_u32(smem_raw) + 1023u) & ~1023u;   // STAGES A slices, then STAGES B slices
    const uint32_t bbase = abase + STAGES * A_BYTES;
    const uint32_t bar0 = smem_u32(bars);
    // barriers: full[s], empty[s], accumulator full[a], accumulator empty[a], drain
    const uint32_t full0 = bar0, empty0 = bar0 + 8 * STAGES, tfull0 = bar0 + 16 * STAGES,
                   tempty0 = tfull0 + 16, drain = tfull0 + 32;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long M = (long)B * SO * SO;
    const int ntiles = (int)((M + BM - 1) / BM);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(full0 + 8 * s, NPROD);
            bar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(tfull0 + 8 * a, 1);
            bar_init(tempty0 + 8 * a, NEPI / 32);
        }
        bar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        flag_s = 0;
    }
    for (int i = tid; i < CO; i += NT) bias_s[i] = bias[i];
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp < 4) {
        // ---- producers: thread tid moves chunk c (8 channels = 16 bytes) of
        // rows r0 + 16 i (i < 8) of A and of rows r0 + 16 j (j < CO / 16) of B;
        // every such row has r mod 8 = r0 mod 8, so one swizzle serves them all
        const int c = tid & 7, r0 = tid >> 3;
        const uint32_t swz = (uint32_t)((c ^ (r0 & 7)) << 4);
        int g = 0;   // stages issued so far (over all tiles)
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            int pix[8], iy0[8], ix0[8];   // pixel (b, 2 oy - 1, 2 ox - 1) of each row; iy0 = S past the end
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const long R = (long)tile * BM + r0 + 16 * i;
                const int b = (int)(R >> (2 * LGSO)), p = (int)(R & (SO * SO - 1));
                const int oy = p >> LGSO, ox = p & (SO - 1);
                iy0[i] = R < M ? 2 * oy - 1 : S;
                ix0[i] = 2 * ox - 1;
                pix[i] = (b * S + 2 * oy - 1) * S + 2 * ox - 1;
            }
            for (int kb = 0; kb < NKB; ++kb, ++g) {
                const int s = g % STAGES;
                if (g >= STAGES && !wait_bar(empty0 + 8 * s, (uint32_t)((g / STAGES - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                const int k0 = kb * BK + 8 * c, tap = k0 >> LGCI, ci0 = k0 & (CI - 1);
                const int ky = tap / 3, kx = tap - 3 * ky;
                const uint32_t sa = abase + s * A_BYTES + swz, sb = bbase + s * B_BYTES + swz;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int iy = iy0[i] + ky, ix = ix0[i] + kx;
                    const bool in = tap < 9 && (unsigned)iy < (unsigned)S && (unsigned)ix < (unsigned)S;
                    const __nv_bfloat16 *src = in ? x + (long)(pix[i] + ky * S + kx) * CI + ci0 : x;
                    cp16_zfill(sa + (r0 + 16 * i) * 128, src, in ? 16u : 0u);
                }
#pragma unroll
                for (int j = 0; j < CO / 16; ++j) {
                    const int co = r0 + 16 * j;
                    cp16_l2(sb + co * 128, w + (long)co * KP + kb * BK + 8 * c);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (g >= LAG) {
                    // stage g - LAG has landed: hand it to the tensor core
                    asm volatile("cp.async.wait_group %0;" ::"n"(LAG) : "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(full0 + 8 * ((g - LAG) % STAGES));
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (ok) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int q = g - LAG > 0 ? g - LAG : 0; q < g; ++q) bar_arrive(full0 + 8 * (q % STAGES));
        }
    } else if (warp < 8) {
        // ---- epilogue: warp 4 + e reads tensor-memory lanes 32 e .. 32 e + 31
        const int e = warp - 4, row = 32 * e + lane;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int a = it & 1;
            const bool got = __all_sync(0xffffffffu, wait_bar(tfull0 + 8 * a, (uint32_t)((it >> 1) & 1), flag));
            if (!got) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long R = (long)tile * BM + row;
#pragma unroll 1
            for (int c0 = 0; c0 < CO; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)(a * CO + c0), v);
                if (R < M) {
                    float f[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) f[j] = fmaxf(__uint_as_float(v[j]) + bias_s[c0 + j], 0.f);
                    if (F32) {
                        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(y) + R * CO + c0);
#pragma unroll
                        for (int q = 0; q < 8; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
                    } else {
                        uint32_t h[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const __nv_bfloat162 t = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
                            h[q] = *reinterpret_cast<const uint32_t *>(&t);
                        }
                        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(y) + R * CO + c0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) dst[q] = make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(tempty0 + 8 * a);
        }
    } else if (lane == 0) {
        // ---- tensor-core issuer
        int g = 0, it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
            const int a = it & 1;
            if (it >= 2 && !wait_bar(tempty0 + 8 * a, (uint32_t)(((it >> 1) - 1) & 1), flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)(a * CO);
            for (int kb = 0; kb < NKB; ++kb, ++g) {
                const int s = g % STAGES;
                if (!wait_bar(full0 + 8 * s, (uint32_t)((g / STAGES) & 1), flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = abase + s * A_BYTES, sb = bbase + s * B_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                        "l"(desc_sw128(sa + kk * 32)), "l"(desc_sw128(sb + kk * 32)), "r"(IDESC), "r"(acc)
                        : "memory");
                }
                commit_to(empty0 + 8 * s);
            }
            if (ok) commit_to(tfull0 + 8 * a);
        }
        // every product issued above completes before the tensor memory is released
        commit_to(drain);
        wait_bar(drain, 0u, flag, false);
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && flag_s) atomicExch(err, 1);
    if (warp == 8) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS));
    }
}

template <int CI, int CO, int S, bool F32>
cudaError_t conv_layer(const __nv_bfloat16 *x, int B, const __nv_bfloat16 *w, const float *bias, void *y, int *err,
                       int num_sms, cudaStream_t st) {
    constexpr size_t smem = cv::smem_bytes(CO);
    auto kern = k_conv_tc<CI, CO, S, F32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long M = (long)B * (S / 2) * (S / 2), tiles = (M + cv::BM - 1) / cv::BM;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    kern<<<grid, cv::NT, smem, st>>>(x, B, w, bias, y, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv_tc(int layer, const void *x, int B, const void *w, const float *bias, void *y, int *err,
                           int num_sms, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    if (num_sms <= 0 || B > (1 << 20) || (reinterpret_cast<uintptr_t>(x) & 15) ||
        (reinterpret_cast<uintptr_t>(w) & 15) || (reinterpret_cast<uintptr_t>(y) & 15))
        return cudaErrorInvalidValue;
    const auto *xb = static_cast<const __nv_bfloat16 *>(x);
    const auto *wb = static_cast<const __nv_bfloat16 *>(w);
    switch (layer) {
        case 1: return conv_layer<32, 64, 64, false>(xb, B, wb, bias, y, err, num_sms, st);
        case 2: return conv_layer<64, 64, 32, false>(xb, B, wb, bias, y, err, num_sms, st);
        case 3: return conv_layer<64, 128, 16, false>(xb, B, wb, bias, y, err, num_sms, st);
        case 4: return conv_layer<128, 128, 8, true>(xb, B, wb, bias, y, err, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}
