// Gnomonic reprojection of the master pattern, shared by the projection
// kernel and the pre-processing kernels that project their input images
// themselves (the same arithmetic: the same pixel values either way).
//
// Paper: "SO(3) Library Generation" (a template is the master pattern seen
// through the detector at an orientation and pattern centre).
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace proj {

// ------------------------------------------------------ Lambert lookup
// Keys' cubic convolution weight, a = -1/2
__device__ __forceinline__ float keys_weight(float t) {
    t = fabsf(t);
    if (t <= 1.f) return (1.5f * t - 2.5f) * t * t + 1.f;
    if (t < 2.f) return ((-0.5f * t + 2.5f) * t - 4.f) * t + 2.f;
    return 0.f;
}

// Rosca equal-area square of a hemisphere, then bilinear (interp 0) or
// bicubic (interp 1, Keys) interpolation of the M x M grid of cell centres,
// clamped at the edges.
__device__ __forceinline__ float master_lookup(const float *__restrict__ master, int M, float x, float y,
                                               float z, int interp = 0) {
    const float az = fabsf(z);
    const float s2 = x * x + y * y;
    float X = 0.f, Y = 0.f;
    if (s2 > 0.f) {
        const float qv = sqrtf(2.f * s2 / (1.f + az));   // sqrt(2 (1 - |z|)), cancellation-free
        const float sp = 0.88622692545275801365f;         // sqrt(pi) / 2
        const float ts = 1.12837916709551257390f;         // 2 / sqrt(pi)
        // the square's sector: |y| <= |x| maps to (sg qv sp, sg qv ts atan(y / x)),
        // else to (sg qv ts atan(x / y), sg qv sp), sg the sign of the larger
        // component; both cases as one division and one arctangent (no divergence)
        const bool xmaj = fabsf(y) <= fabsf(x);
        const float num = xmaj ? y : x, den = xmaj ? x : y;
        const float sg = den >= 0.f ? 1.f : -1.f;
        const float u = sg * qv * sp, t = sg * qv * ts * atanf(num / den);
        X = xmaj ? u : t;
        Y = xmaj ? t : u;
    }
    const float invL = 0.79788456080286535588f;           // 1 / sqrt(pi / 2)
    float fx = (X * invL + 1.f) * (0.5f * M) - 0.5f;
    float fy = (Y * invL + 1.f) * (0.5f * M) - 0.5f;
    fx = fminf(fmaxf(fx, 0.f), (float)(M - 1));
    fy = fminf(fmaxf(fy, 0.f), (float)(M - 1));
    if (interp == 1) {
        const float *g = master + (z >= 0.f ? 0 : (size_t)M * M);
        const int i0 = (int)floorf(fx), j0 = (int)floorf(fy);
        float s = 0.f;
#pragma unroll
        for (int dj = -1; dj <= 2; ++dj) {
            const int j = min(max(j0 + dj, 0), M - 1);
            const float wy = keys_weight(fy - (float)(j0 + dj));
            float row = 0.f;
#pragma unroll
            for (int di = -1; di <= 2; ++di) {
                const int i = min(max(i0 + di, 0), M - 1);
                row = fmaf(keys_weight(fx - (float)(i0 + di)), __ldg(g + (size_t)j * M + i), row);
            }
            s = fmaf(wy, row, s);
        }
        return s;
    }
    int i0 = min((int)floorf(fx), M - 2), j0 = min((int)floorf(fy), M - 2);
    const float tx = fx - i0, ty = fy - j0;
    const float *g = master + (z >= 0.f ? 0 : (size_t)M * M) + (size_t)j0 * M + i0;
    const float a = __ldg(g), b = __ldg(g + 1), c = __ldg(g + M), d = __ldg(g + M + 1);
    return (1.f - ty) * ((1.f - tx) * a + tx * b) + ty * ((1.f - tx) * c + tx * d);
}

// per-image frame: G = R(q) Rx(alpha) (detector direction -> crystal
// direction) and the pattern centre in pixels, in FP32 (FP64 here stalled
// the block on GB300's narrow FP64 pipe)
struct Frame {
    float G[9];
    float pc[3];
};
__device__ __forceinline__ void frame(const double *__restrict__ q4, const double *__restrict__ pc3,
                                      const ProjArgs &a, Frame &f) {
    float w = (float)q4[0], x = (float)q4[1], y = (float)q4[2], z = (float)q4[3];
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    float R[9];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
    const float sa = (float)a.sa, ca = (float)a.ca;
    for (int i = 0; i < 3; ++i) {
        f.G[3 * i + 0] = R[3 * i + 0];
        f.G[3 * i + 1] = R[3 * i + 1] * ca + R[3 * i + 2] * sa;
        f.G[3 * i + 2] = -R[3 * i + 1] * sa + R[3 * i + 2] * ca;
    }
    double px = a.pcx, py = a.pcy, pz = a.pcz;
    if (pc3) { px = pc3[0]; py = pc3[1]; pz = pc3[2]; }
    f.pc[0] = (float)px * (float)a.W;
    f.pc[1] = (float)py * (float)a.H;
    f.pc[2] = (float)pz * (float)a.W;
}
// the part of a pixel's detector direction that depends on its column j alone
// (detector column ox + j): the x offset from the pattern centre and the
// rotated contributions of the x and z components, G[:, 0] dx + G[:, 2] dz
struct Col {
    float dx, bx, by, bz;
};
__device__ __forceinline__ Col column(const Frame &f, const ProjArgs &a, int j) {
    const float dx = (float)(a.ox + j) + 0.5f - f.pc[0], dz = f.pc[2];
    return Col{dx, fmaf(f.G[0], dx, f.G[2] * dz), fmaf(f.G[3], dx, f.G[5] * dz), fmaf(f.G[6], dx, f.G[8] * dz)};
}
// the template's value at pixel (i, c) of the output region (detector pixel
// (oy + i, ox + j) for the column c = column(f, a, j), centre of the pixel):
// the crystal direction G d / |d| (G is a rotation, so the direction is
// rotated first and normalised after) looked up in the master pattern
__device__ __forceinline__ float pixel(const Frame &f, const Col &c, const float *__restrict__ master, int M,
                                       const ProjArgs &a, int i) {
    const float dy = f.pc[1] - ((float)(a.oy + i) + 0.5f), dz = f.pc[2];
    const float inv = rsqrtf(fmaf(dy, dy, fmaf(c.dx, c.dx, dz * dz)));
    const float cx = fmaf(f.G[1], dy, c.bx) * inv;
    const float cy = fmaf(f.G[4], dy, c.by) * inv;
    const float cz = fmaf(f.G[7], dy, c.bz) * inv;
    return master_lookup(master, M, cx, cy, cz, a.interp);
}
__device__ __forceinline__ float pixel(const Frame &f, const float *__restrict__ master, int M, const ProjArgs &a,
                                       int i, int j) {
    return pixel(f, column(f, a, j), master, M, a, i);
}

}  // namespace proj
