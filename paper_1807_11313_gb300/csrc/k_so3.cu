// SO(3) sampling (paper: "SO(3) Library Generation", "SO(3) Sampling
// Frequency", the second Eq. 6, Fig. 2): the S^2 x S^1 library generator in
// the cubic fundamental zone and the nearest-neighbour disorientation study.
//
// k_so3_points: one thread per grid point (ring, azimuth, S^1 step) -> Bunge
//   quaternion in FP64 and its fundamental-zone flag.
// k_block_count / k_scan_blocks / k_compact: order-preserving compaction of
//   the flagged points (per-block counts, one-CTA exclusive scan, scatter).
// k_nn_partial: nearest neighbour under the 24 cubic rotations.  For
//   m = a b^-1 the largest |scalar part| of S m over the group is
//   max(t1, (t1 + t2) / sqrt 2, (t1 + t2 + t3 + t4) / 2), t the sorted
//   absolute components of m (identity and the 180-degree axis rotations, the
//   90-degree and <110> rotations, the 120-degree <111> rotations).  FP32
//   per pair, the best (largest |w|, lowest index) packed into a 64-bit key
//   and merged across qb slices with atomicMax; k_nn_finish recomputes the
//   chosen pair's angle in FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kNnThreads = 128, kNnTile = 1024;

// a quaternion (w, x, y, z) held as members (x, y, z, w) = (w, x, y, z) in order
struct Qd {
    double x, y, z, w;
};
__device__ __forceinline__ Qd make_qd(double a, double b, double c, double d) { return Qd{a, b, c, d}; }
__device__ __forceinline__ Qd qmul_d(Qd a, Qd b) {
    return make_qd(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                   a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y, a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

__global__ void k_so3_points(const long long *__restrict__ ring_start, int n_rings, int n_polar, int n_s1,
                             const int *__restrict__ ring_az, long long G, double *__restrict__ q_all,
                             int *__restrict__ flag) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    int lo = 0, hi = n_rings - 1;   // last ring with ring_start <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ring_start[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int i = lo, na = ring_az[i];
    const long long r = g - ring_start[i];
    const int j = (int)(r / n_s1), k = (int)(r % n_s1);
    const double Phi = XCF_PI * i / n_polar;
    const double p1 = 2 * XCF_PI * (j + 0.5 * (i % 2)) / na, p2 = 2 * XCF_PI * k / n_s1;
    double s1, c1, s2, c2, s3, c3;
    sincos(0.5 * p1, &s1, &c1);
    sincos(0.5 * Phi, &s2, &c2);
    sincos(0.5 * p2, &s3, &c3);
    Qd q = qmul_d(qmul_d(make_qd(c1, 0, 0, s1), make_qd(c2, s2, 0, 0)), make_qd(c3, 0, 0, s3));
    double nq = sqrt(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    if (q.x < 0) nq = -nq;
    q = make_qd(q.x / nq, q.y / nq, q.z / nq, q.w / nq);
    const double w = q.x > 1e-300 ? q.x : 1e-300;
    const double r0 = fabs(q.y) / w, r1 = fabs(q.z) / w, r2 = fabs(q.w) / w;
    const double mx = fmax(r0, fmax(r1, r2));
    flag[g] = (mx <= sqrt(2.0) - 1.0 + 1e-12 && r0 + r1 + r2 <= 1.0 + 1e-12) ? 1 : 0;
    double *o = q_all + 4 * g;
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
}

constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
    // exclusive scan over the block (kScanBlock threads)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kScanBlock / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;   // inclusive warp totals
    }
    __syncthreads();
    const int before = warp ? sh[warp - 1] : 0;
    if (total) *total = sh[kScanBlock / 32 - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_block_count(const int *__restrict__ flag, long long G,
                                                            int *__restrict__ counts) {
    __shared__ int sh[32];
    const long long g = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    int total;
    block_excl_scan(g < G ? flag[g] : 0, sh, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// exclusive scan of nb block counts in place (one CTA, serial over chunks); total -> *out_total
__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(int *__restrict__ counts, int nb,
                                                            long long *__restrict__ out_total) {
    __shared__ int sh[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanBlock) {
        const int i = base + threadIdx.x;
        int total;
        const int ex = block_excl_scan(i < nb ? counts[i] : 0, sh, &total);
        const long long c = carry;
        if (i < nb) counts[i] = (int)(c + ex);
        __syncthreads();
        if (threadIdx.x == 0) carry = c + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_compact(const double *__restrict__ q_in, const int *__restrict__ flag,
                                                        long long G, const int *__restrict__ offsets,
                                                        double *__restrict__ q_out) {
    __shared__ int sh[32];
    const long long g = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int f = g < G ? flag[g] : 0;
    const int ex = block_excl_scan(f, sh, nullptr);
    if (f) {
        const long long o = (long long)offsets[blockIdx.x] + ex;
        for (int c = 0; c < 4; ++c) q_out[4 * o + c] = q_in[4 * g + c];
    }
}

__device__ __forceinline__ float cubic_max_w(float4 m) {
    float a = fabsf(m.x), b = fabsf(m.y), c = fabsf(m.z), d = fabsf(m.w);
    // two largest of four
    const float hi1 = fmaxf(a, b), lo1 = fminf(a, b), hi2 = fmaxf(c, d), lo2 = fminf(c, d);
    const float t1 = fmaxf(hi1, hi2), t2 = fmaxf(fminf(hi1, hi2), fmaxf(lo1, lo2));
    return fmaxf(t1, fmaxf((t1 + t2) * 0.70710678118654752f, 0.5f * (a + b + c + d)));
}

// m = a conj(b), (w, x, y, z) in (x, y, z, w)
__device__ __forceinline__ float4 qmul_conj_f(float4 a, float4 b) {
    return make_float4(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w, -a.x * b.y + a.y * b.x - a.z * b.w + a.w * b.z,
                       -a.x * b.z + a.y * b.w + a.z * b.x - a.w * b.y, -a.x * b.w - a.y * b.z + a.z * b.y + a.w * b.x);
}

// grid (ceil(na / kNnThreads), slices): thread = one qa, slice = a range of qb
__global__ void __launch_bounds__(kNnThreads) k_nn_partial(const double *__restrict__ qa, int na,
                                                           const double *__restrict__ qb, int nb, int mode,
                                                           int per_slice, unsigned long long *__restrict__ keys) {
    __shared__ float4 tile[kNnTile];
    const int i = blockIdx.x * kNnThreads + threadIdx.x;
    const int j0 = blockIdx.y * per_slice, j1 = min(nb, j0 + per_slice);
    float4 a = make_float4(1.f, 0.f, 0.f, 0.f);
    if (i < na) a = make_float4((float)qa[4 * i], (float)qa[4 * i + 1], (float)qa[4 * i + 2], (float)qa[4 * i + 3]);
    float bw = -1.f;
    int bj = -1;
    for (int t0 = j0; t0 < j1; t0 += kNnTile) {
        const int tn = min(kNnTile, j1 - t0);
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += kNnThreads) {
            const double *b = qb + 4 * (size_t)(t0 + t);
            tile[t] = make_float4((float)b[0], (float)b[1], (float)b[2], (float)b[3]);
        }
        __syncthreads();
        if (i >= na) continue;
        const int lim = mode == 2 ? min(tn, i - t0) : tn;   // mode 2: j < i only
        for (int t = 0; t < lim; ++t) {
            if (mode == 1 && t0 + t == i) continue;
            const float w = cubic_max_w(qmul_conj_f(a, tile[t]));
            if (w > bw) { bw = w; bj = t0 + t; }   // ascending j: ties keep the lowest
        }
    }
    if (i < na && bj >= 0) {
        // larger w first; among equal w the lower index (larger complement)
        const unsigned long long key = ((unsigned long long)__float_as_uint(bw) << 32) | (0xffffffffu - (unsigned)bj);
        atomicMax(keys + i, key);
    }
}

__global__ void k_nn_finish(const double *__restrict__ qa, int na, const double *__restrict__ qb,
                            const unsigned long long *__restrict__ keys, double *__restrict__ angle,
                            int *__restrict__ index) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const unsigned long long k = keys[i];
    if (k == 0) { angle[i] = -1.0; index[i] = -1; return; }
    const int j = (int)(0xffffffffu - (unsigned)(k & 0xffffffffu));
    const Qd a = make_qd(qa[4 * i], qa[4 * i + 1], qa[4 * i + 2], qa[4 * i + 3]);
    const Qd b = make_qd(qb[4 * (size_t)j], -qb[4 * (size_t)j + 1], -qb[4 * (size_t)j + 2], -qb[4 * (size_t)j + 3]);
    const Qd m = qmul_d(a, b);
    const double nm = sqrt(m.x * m.x + m.y * m.y + m.z * m.z + m.w * m.w);
    double t[4] = {fabs(m.x) / nm, fabs(m.y) / nm, fabs(m.z) / nm, fabs(m.w) / nm};
    for (int p = 0; p < 3; ++p)   // sort descending
        for (int q = 0; q < 3 - p; ++q)
            if (t[q] < t[q + 1]) { const double s = t[q]; t[q] = t[q + 1]; t[q + 1] = s; }
    double w = fmax(t[0], fmax((t[0] + t[1]) * 0.70710678118654752440, 0.5 * (t[0] + t[1] + t[2] + t[3])));
    if (w > 1.0) w = 1.0;
    angle[i] = 2.0 * acos(w) * 180.0 / XCF_PI;
    index[i] = j;
}

__global__ void k_keep_flags(const double *__restrict__ angle, long long n, double thr, int *__restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (angle[i] >= 0.0 && angle[i] < thr) ? 0 : 1;
}

}  // namespace

cudaError_t launch_keep_flags(const double *angle, long long n, double thr, int *flag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_keep_flags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(angle, n, thr, flag);
    return cudaGetLastError();
}

cudaError_t launch_so3_points(const long long *ring_start, int n_rings, int n_polar, int n_s1, const int *ring_az,
                              long long G, double *q_all, int *flag, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    k_so3_points<<<(unsigned)((G + 255) / 256), 256, 0, st>>>(ring_start, n_rings, n_polar, n_s1, ring_az, G, q_all,
                                                              flag);
    return cudaGetLastError();
}

int compact_blocks(long long G) { return (int)((G + kScanBlock - 1) / kScanBlock); }

cudaError_t launch_compact(const double *q_in, const int *flag, long long G, int *block_counts, long long *total,
                           double *q_out, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    const int nb = compact_blocks(G);
    k_block_count<<<nb, kScanBlock, 0, st>>>(flag, G, block_counts);
    k_scan_blocks<<<1, kScanBlock, 0, st>>>(block_counts, nb, total);
    if (q_out) k_compact<<<nb, kScanBlock, 0, st>>>(q_in, flag, G, block_counts, q_out);
    return cudaGetLastError();
}

cudaError_t launch_nearest_disorientation(const double *qa, int na, const double *qb, int nb, int mode,
                                          unsigned long long *keys, double *angle, int *index, int num_sms,
                                          cudaStream_t st) {
    if (na <= 0) return cudaSuccess;
    if (nb < 0 || mode < 0 || mode > 2) return cudaErrorInvalidValue;
    const int gx = (na + kNnThreads - 1) / kNnThreads;
    // enough slices of qb for four CTAs per SM, each slice at least one tile
    int slices = (4 * num_sms + gx - 1) / gx;
    const int max_slices = nb > 0 ? (nb + kNnTile - 1) / kNnTile : 1;
    if (slices > max_slices) slices = max_slices;
    if (slices < 1) slices = 1;
    if (slices > 65535) slices = 65535;
    const int per = nb > 0 ? (nb + slices - 1) / slices : 1;
    cudaError_t e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * na, st);
    if (e != cudaSuccess) return e;
    if (nb > 0) k_nn_partial<<<dim3(gx, slices), kNnThreads, 0, st>>>(qa, na, qb, nb, mode, per, keys);
    k_nn_finish<<<(na + 127) / 128, 128, 0, st>>>(qa, na, qb, keys, angle, index);
    return cudaGetLastError();
}
