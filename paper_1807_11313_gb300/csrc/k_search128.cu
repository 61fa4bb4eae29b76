// All-pairs XCF search for 128 x 128 detectors (the hot loop of the indexer).
//
// Paper: Eqs. 3 and 6 (correlation surface r(s) = sum_k conj(S_t) S_p
// exp(+2 pi i k.s / N)), Fig. 1 B-C (best template by peak height), Fig. 5 /
// Discussion (one inverse FFT per pattern-template pair dominates the cost).
//
// One CTA (512 threads, one per SM) keeps one pattern's half spectrum in
// shared memory and streams the library's half spectra from L2/HBM, two
// templates per inverse FFT: Z = X1 + i X2 with X_j = conj(S_tj) S_p extended
// to the full spectrum by Hermitian symmetry, so that Re(IFFT Z) and
// Im(IFFT Z) are the two real correlation surfaces.  The 128 x 128 inverse FFT
// runs in three register rounds separated by two shared-memory transposes
// (rows y = k2 + 16 k1 of the column transform, columns x = k3 + 4 k4 of the
// row transform):
//   round 1: thread (q, l) owns stored column q and rows u = l + 8m: two
//            16-point FFTs over m (of X1 and X2), twiddle W128^(l k2); the
//            conjugate-symmetric partner column 128 - q is written from the
//            same registers (conj(A1) + i conj(A2) at sub-sequence 8 - l);
//   round 2: thread (k2, g): radix-8 over l completes the column transform
//            for rows k2 + 16 k1, then radix-4 over the columns g + 32 i and
//            twiddle W128^(g k3);
//   round 3: thread (y, k3): a 32-point FFT over g gives row y, columns
//            k3 + 4 k4, of both surfaces; the max of each is reduced.
// Each thread holds 32 complex values per round (at most 128 registers), so
// sixteen warps share an SM and hide one another's shared-memory latency.
// No surface is written to global memory; only the per-pattern best key (and
// optionally every per-pair peak) leave the kernel.
//
// Library spectra are read in a packed "search layout" (pack_search_layout):
// for each template, columns 0..63 as [l][m/2][q][m&1] with u = l + 8m (64 KB,
// so that the 16 rows a round-1 thread needs are 8 conflict-free 16-byte
// shared loads), then column 64.  The next pair is copied from L2 with
// cp.async while round 3 computes: round 3 first pulls its values into
// registers, after which the transpose buffer (128 KB) holds exactly columns
// 0..63 of two templates.
#include "common.cuh"
#include "kernels.cuh"

#include "search128.cuh"

namespace {

using namespace s128;

__global__ void __launch_bounds__(NT, 1)
k_search128(const float2 *__restrict__ Spk, int T, const float2 *__restrict__ Sp,
            const int *__restrict__ degen, int pairs_per_cta,
            unsigned long long *__restrict__ keys, float *__restrict__ peaks_all) {
    const int p = blockIdx.y;
    if (degen[p]) return;
    const int npairs = (T + 1) / 2;
    const int pb = blockIdx.x * pairs_per_cta;
    const int pe = min(npairs, pb + pairs_per_cta);
    if (pb >= pe) return;
    search_body(Spk, T, Sp, p, pb, pe, keys, peaks_all);
}

// standard half spectra [T][128][65] -> packed search layout [T][8320]
__global__ void k_pack_search_layout(const float2 *__restrict__ src, int T, float2 *__restrict__ dst) {
    const size_t total = (size_t)T * SPEC;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t t = i / SPEC;
        const int k = (int)(i % SPEC), u = k / HW, v = k % HW;
        dst[t * SPEC + (v < 64 ? pk(u, v) : COL64 + u)] = src[i];
    }
}

}  // namespace

cudaError_t launch_pack_search_layout(const float2 *spectra, int T, int N_, float2 *packed, cudaStream_t st) {
    if (N_ == 256) return launch_pack_c256(spectra, T, packed, st);
    if (N_ != N) return cudaErrorInvalidValue;
    if (T <= 0) return cudaSuccess;
    const size_t total = (size_t)T * SPEC;
    const int blocks = (int)((total + 255) / 256 < 65536 ? (total + 255) / 256 : 65536);
    k_pack_search_layout<<<blocks, 256, 0, st>>>(spectra, T, packed);
    return cudaGetLastError();
}

cudaError_t launch_search128(const float2 *Spk, int T, const float2 *Sp, const int *degen, int P,
                             unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_search128, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int npairs = (T + 1) / 2;
    // one CTA per SM at a time: split the library into at most max(4, SMs / P)
    // parts of at least 8 pairs each, taking the part count c that minimises
    // waves(P c) x pairs per part (the split does not change the results: the
    // key is an exact maximum, the lowest template winning ties)
    const int cap = max(1, min(max(4, (num_sms + P - 1) / P), (npairs + 7) / 8));
    int chunks = 1;
    long best_cost = -1;
    for (int c = 1; c <= cap; ++c) {
        const long waves = ((long)P * c + num_sms - 1) / num_sms;
        const long cost = waves * ((npairs + c - 1) / c);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            chunks = c;
        }
    }
    int ppc = (npairs + chunks - 1) / chunks;
    chunks = (npairs + ppc - 1) / ppc;
    dim3 grid(chunks, P);
    k_search128<<<grid, NT, SMEM_BYTES, st>>>(Spk, T, Sp, degen, ppc, keys, peaks_all);
    return cudaGetLastError();
}
