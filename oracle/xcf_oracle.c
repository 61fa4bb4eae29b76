/*
 * FP64 CPU oracle for the refined template-matching EBSD indexer
 * (Foden, Collins, Wilkinson & Britton, arXiv 1807.11313).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  It is used by the tests, by
 * __graft_entry__.smoke() and by the CPU-baseline leg of bench.py, and by
 * nothing else.  It shares no code, header, table or constant with the CUDA
 * library: it has its own DFT/FFT, its own Lambert map, its own projector.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent or garbled the reading taken is stated in the comment.
 * Parity unpinned: the window shape, the band-pass shape and its cut-offs, the
 * log-polar sampling constants and the refinement's sign conventions are not
 * fixed by the paper (it gives no values); they are pinned only against the
 * paper's qualitative statements and internal invariants.  The implementation
 * of those readings is pinned to library routines (scipy's periodic Hann,
 * products of Fourier-domain Gaussians, bilinear resampling, numpy's FFT).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------------- */
/* options and geometry                                                    */
/* ---------------------------------------------------------------------- */
typedef struct {
    int32_t window;      /* 0 = none, 1 = periodic Hann (separable)           */
    double sigma_hp;     /* Gaussian high-pass sigma, cycles per image         */
    double sigma_lp;     /* Gaussian low-pass sigma, cycles per image          */
    int32_t lp_nr;       /* log-polar radial samples                           */
    int32_t lp_neta;     /* log-polar angular samples                          */
    double lp_rmin;      /* smallest radius, pixels                            */
    double lp_rmax;      /* largest radius, pixels                             */
    int32_t upsample;    /* 0: 3-point parabola; U >= 2: up-sampled peak       */
    int32_t interp;      /* master lookup: 0 bilinear, 1 bicubic (Keys)        */
    double ndp_bg_sigma; /* NDP background: Gaussian sigma, px; 0 = n/8, < 0 off */
    int32_t lp_windows;  /* log-polar radial windows of the Z step (<= 1: one)  */
} orc_opts;

typedef struct {
    int32_t width, height;       /* detector pixels                            */
    double pcx, pcy, pcz;        /* Bruker-style pattern centre                */
    double sample_tilt_deg;      /* sample tilt (70 deg in the paper)          */
    double detector_tilt_deg;
} orc_geom;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Fourier transforms (Eq. 4)                                              */
/* ---------------------------------------------------------------------- */

/* Direct O(n^2) 1-D DFT: out[k] = sum_x in[x] exp(sign 2 pi i k x / n).
 * Unscaled.  The reference the FFT below is pinned against. */
void orc_dft1(const cplx *in, cplx *out, int n, int sign) {
    for (int k = 0; k < n; ++k) {
        cplx s = 0;
        for (int x = 0; x < n; ++x) {
            double a = sign * 2.0 * ORC_PI * (double)(((long)k * x) % n) / n;
            s += in[x] * (cos(a) + I * sin(a));
        }
        out[k] = s;
    }
}

/* Direct O(n^4) 2-D DFT of an n x n array (row-major), unscaled. */
void orc_dft2_brute(const cplx *in, cplx *out, int n, int sign) {
    for (int u = 0; u < n; ++u)
        for (int v = 0; v < n; ++v) {
            cplx s = 0;
            for (int x = 0; x < n; ++x)
                for (int y = 0; y < n; ++y) {
                    long p = ((long)u * x + (long)v * y) % n;
                    double a = sign * 2.0 * ORC_PI * (double)p / n;
                    s += in[x * n + y] * (cos(a) + I * sin(a));
                }
            out[u * n + v] = s;
        }
}

/* In-place iterative radix-2 Cooley-Tukey FFT of length n (a power of two),
 * stride `st` between elements.  Unscaled; sign -1 forward, +1 inverse. */
static void fft1_strided(cplx *x, int n, int st, int sign) {
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i * st];
            x[i * st] = x[j * st];
            x[j * st] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < len / 2; ++k) {
                double a = sign * 2.0 * ORC_PI * k / len;
                cplx w = cos(a) + I * sin(a);
                cplx u = x[(i + k) * st];
                cplx v = x[(i + k + len / 2) * st] * w;
                x[(i + k) * st] = u + v;
                x[(i + k + len / 2) * st] = u - v;
            }
        }
    }
}

/* A line of any length: the radix-2 FFT for powers of two, the direct DFT
 * (orc_dft1) otherwise (the 96- and 160-pixel native detectors). */
static void line_transform(cplx *x, int n, int st, int sign) {
    if (n <= 0) return;
    if ((n & (n - 1)) == 0) {
        fft1_strided(x, n, st, sign);
        return;
    }
    cplx *a = malloc(sizeof(cplx) * n), *b = malloc(sizeof(cplx) * n);
    if (!a || !b) abort();   /* test infrastructure: no recovery from an exhausted host */
    for (int i = 0; i < n; ++i) a[i] = x[(long)i * st];
    orc_dft1(a, b, n, sign);
    for (int i = 0; i < n; ++i) x[(long)i * st] = b[i];
    free(a); free(b);
}

void orc_fft1(cplx *x, int n, int sign) { line_transform(x, n, 1, sign); }

/* 2-D transform of an n x n row-major array: rows, then columns.  Unscaled. */
void orc_fft2(cplx *x, int n, int sign) {
    for (int r = 0; r < n; ++r) line_transform(x + (long)r * n, n, 1, sign);
    for (int c = 0; c < n; ++c) line_transform(x + c, n, n, sign);
}

/* ---------------------------------------------------------------------- */
/* pre-processing (Eq. 4 and the filtering / windowing of the FFT method)  */
/* ---------------------------------------------------------------------- */

/* Centred crop of a W x H detector to the largest 2^k square side (<= cap):
 * the paper crops to a 2^n x 2^n field of view and updates the PC so that it
 * keeps pointing at the same pixel (footnotes 1-2 of the FFT section; the
 * worked example 200 -> 128 px moves PCx 0.4 -> 0.34).  Outputs the square
 * side n, the crop offsets and the updated PC.  Returns 0, or -1 if the side
 * would be below 16. */
int orc_crop_ex(int W, int H, int cap, int native, double pcx, double pcy, double pcz,
                int *n_out, int *off_x, int *off_y, double pc_out[3]);
int orc_crop(int W, int H, int cap, double pcx, double pcy, double pcz,
             int *n_out, int *off_x, int *off_y, double pc_out[3]) {
    return orc_crop_ex(W, H, cap, 0, pcx, pcy, pcz, n_out, off_x, off_y, pc_out);
}

/* The crop with native sides (native != 0): the largest side of
 * {16, 32, 64, 96, 128, 160, 200, 256} that fits, so that 96-, 160- and
 * 200-pixel detectors are used whole (the paper crops to 2^n only because its
 * FFT and filters are easier there, footnote 1 of the FFT section). */
int orc_crop_ex(int W, int H, int cap, int native, double pcx, double pcy, double pcz,
                int *n_out, int *off_x, int *off_y, double pc_out[3]) {
    static const int sides[8] = {16, 32, 64, 96, 128, 160, 200, 256};
    int m = W < H ? W : H;
    int n = 1;
    if (native) {
        n = 0;
        for (int i = 0; i < 8; ++i)
            if (sides[i] <= m && sides[i] <= cap) n = sides[i];
    } else {
        while (n * 2 <= m && n * 2 <= cap) n *= 2;
    }
    if (n < 16) return -1;
    int ox = (W - n) / 2, oy = (H - n) / 2;
    *n_out = n; *off_x = ox; *off_y = oy;
    pc_out[0] = (pcx * W - ox) / n;
    pc_out[1] = (pcy * H - oy) / n;
    pc_out[2] = pcz * W / n;      /* detector distance in pixels is unchanged */
    return 0;
}

/* Band-pass filter H(u,v) at integer frequency (u, v) of an n x n transform:
 * the paper uses a high-pass (background) and a low-pass (noise) filter in
 * Fourier space without giving their form; reading: Gaussian high-pass times
 * Gaussian low-pass on the radial signed frequency rho. */
double orc_bandpass(int u, int v, int n, double sigma_hp, double sigma_lp) {
    double fu = (u < n / 2) ? u : u - n;
    double fv = (v < n / 2) ? v : v - n;
    double rho2 = fu * fu + fv * fv;
    double hp = 1.0 - exp(-rho2 / (2.0 * sigma_hp * sigma_hp));
    double lp = exp(-rho2 / (2.0 * sigma_lp * sigma_lp));
    return hp * lp;
}

/* Window: the paper manages wrap-around artefacts with a window of unstated
 * type; reading: separable periodic Hann, w(k) = (1 - cos(2 pi k / n)) / 2. */
double orc_window(int k, int n, int kind) {
    if (kind == 0) return 1.0;
    return 0.5 * (1.0 - cos(2.0 * ORC_PI * k / n));
}

/* Pre-process one n x n image (already cropped):
 *   1. contrast normalisation to zero mean, unit standard deviation (the
 *      paper's simulations fix mean 0 and std 1 for both templates and
 *      experimental patterns);
 *   2. windowing;
 *   3. unitary 2-D DFT (Eq. 4);
 *   4. band-pass filter;
 *   5. division by the norm of the filtered spectrum, so that the
 *      correlation at zero shift of an image with itself is 1 and correlation
 *      coefficients are comparable across templates (normalisation by the
 *      autocorrelations of F and G, FFT section).
 * S receives the full n x n spectrum; if y is non-NULL it receives the
 * filtered spatial image y = unitary inverse DFT of S (real part), which has
 * unit L2 norm.  Returns 0, or 1 if the image is degenerate (zero variance or
 * zero filtered energy), in which case S (and y) are zero. */
int orc_prep(const double *img, int n, const orc_opts *o, cplx *S, double *y) {
    long nn = (long)n * n;
    double mean = 0.0;
    for (long i = 0; i < nn; ++i) mean += img[i];
    mean /= nn;
    double var = 0.0;
    for (long i = 0; i < nn; ++i) var += (img[i] - mean) * (img[i] - mean);
    var /= nn;
    double sd = sqrt(var);
    if (!(sd > 1e-12 * (1.0 + fabs(mean)))) {
        memset(S, 0, sizeof(cplx) * nn);
        if (y) memset(y, 0, sizeof(double) * nn);
        return 1;
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c)
            S[(long)r * n + c] = (img[(long)r * n + c] - mean) / sd *
                                 orc_window(r, n, o->window) * orc_window(c, n, o->window);
    orc_fft2(S, n, -1);
    double energy = 0.0;
    for (int u = 0; u < n; ++u)
        for (int v = 0; v < n; ++v) {
            long k = (long)u * n + v;
            S[k] = S[k] / n * orc_bandpass(u, v, n, o->sigma_hp, o->sigma_lp);
            energy += creal(S[k]) * creal(S[k]) + cimag(S[k]) * cimag(S[k]);
        }
    if (!(energy > 0.0)) {
        memset(S, 0, sizeof(cplx) * nn);
        if (y) memset(y, 0, sizeof(double) * nn);
        return 1;
    }
    double inv = 1.0 / sqrt(energy);
    for (long k = 0; k < nn; ++k) S[k] *= inv;
    if (y) {
        cplx *tmp = malloc(sizeof(cplx) * nn);
        memcpy(tmp, S, sizeof(cplx) * nn);
        orc_fft2(tmp, n, +1);
        for (long k = 0; k < nn; ++k) y[k] = creal(tmp[k]) / n;
        free(tmp);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* cross-correlation (Eqs. 2, 3, 6)                                        */
/* ---------------------------------------------------------------------- */

/* Correlation surface r(s) = sum_k conj(St[k]) Sp[k] exp(+2 pi i k.s / n)
 * (Eq. 6 with the conjugate on the template; Eq. 3 omits it).  With unit-norm
 * spectra this is the normalised correlation coefficient, r(s) in [-1, 1];
 * r is maximal at s = d when the pattern is the template translated by +d. */
void orc_xcf_surface(const cplx *St, const cplx *Sp, int n, double *r) {
    long nn = (long)n * n;
    cplx *X = malloc(sizeof(cplx) * nn);
    for (long k = 0; k < nn; ++k) X[k] = conj(St[k]) * Sp[k];
    orc_fft2(X, n, +1);
    for (long k = 0; k < nn; ++k) r[k] = creal(X[k]);
    free(X);
}

/* Brute-force circular spatial cross-correlation (Eq. 2 with indices taken
 * modulo n): r(m, l) = sum_{i,j} a[i, j] b[i + m, j + l]. */
void orc_xcf_spatial(const double *a, const double *b, int n, double *r) {
    for (int m = 0; m < n; ++m)
        for (int l = 0; l < n; ++l) {
            double s = 0.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    s += a[i * n + j] * b[((i + m) % n) * n + (j + l) % n];
            r[m * n + l] = s;
        }
}

/* 3-point parabolic vertex offset, clamped to [-0.5, 0.5]; 0 if not a maximum.
 * The paper up-samples the peak for a sub-pixel shift without giving the
 * method; reading: a parabola through the peak and its two neighbours. */
double orc_parabola(double cm, double c0, double cp) {
    double den = cm - 2.0 * c0 + cp;
    if (!(den < 0.0)) return 0.0;
    double d = (cm - cp) / (2.0 * den);
    if (d > 0.5) d = 0.5;
    if (d < -0.5) d = -0.5;
    return d;
}

/* Peak of a correlation surface: integer argmax (ties -> lowest row-major
 * index), value, and sub-pixel shift (dx, dy) = wrapped integer shift plus the
 * parabolic offsets along columns and rows, wrapped into [-n/2, n/2). */
void orc_peak(const double *r, int n, double *peak, int *sy, int *sx,
              double *dx, double *dy) {
    long nn = (long)n * n, best = 0;
    for (long k = 1; k < nn; ++k)
        if (r[k] > r[best]) best = k;
    int y0 = (int)(best / n), x0 = (int)(best % n);
    double c0 = r[best];
    double cxm = r[(long)y0 * n + (x0 + n - 1) % n], cxp = r[(long)y0 * n + (x0 + 1) % n];
    double cym = r[(long)((y0 + n - 1) % n) * n + x0], cyp = r[(long)((y0 + 1) % n) * n + x0];
    *peak = c0;
    *sy = y0;
    *sx = x0;
    *dx = (x0 < n / 2 ? x0 : x0 - n) + orc_parabola(cxm, c0, cxp);
    *dy = (y0 < n / 2 ? y0 : y0 - n) + orc_parabola(cym, c0, cyp);
}

/* Up-sampled peak (the paper's sub-pixel "up-sampling", its reference [17]
 * absent; reading: the correlation evaluated off the integer grid by its
 * Fourier series, as in matrix-multiply DFT up-sampling).  X = conj(St) Sp is
 * the full n x n cross-power spectrum; the real surface off the grid is taken
 * as r(y, x) = sum over stored columns v = 0..n/2 of w_v Re sum_u X[u][v]
 * exp(+2 pi i (f(u) y + v x) / n), w_0 = w_{n/2} = 1, w_v = 2 otherwise, f(u)
 * the signed frequency (u, or u - n above n/2); at integer (y, x) it is the
 * FFT surface.  It is evaluated on the grid y0 + (m - U)/U, x0 + (l - U)/U,
 * m, l = 0..2U (+-1 px around the integer argmax (y0, x0) of r), and the grid
 * argmax (ties -> lowest (m, l) row-major) gives the peak and the shift
 * (wrapped integer shift plus the grid offsets). */
void orc_peak_upsampled(const cplx *X, const double *r, int n, int U, double *peak, double *dx, double *dy) {
    long nn = (long)n * n, best = 0;
    for (long k = 1; k < nn; ++k)
        if (r[k] > r[best]) best = k;
    int y0 = (int)(best / n), x0 = (int)(best % n), M = 2 * U + 1, H = n / 2 + 1;
    cplx *T1 = malloc(sizeof(cplx) * M * H);
    for (int m = 0; m < M; ++m) {
        double y = y0 + (double)(m - U) / U;
        for (int v = 0; v < H; ++v) {
            cplx acc = 0;
            for (int u = 0; u < n; ++u) {
                double fu = u < n / 2 ? u : u - n;
                double a = 2.0 * ORC_PI * fu * y / n;
                acc += X[(long)u * n + v] * (cos(a) + I * sin(a));
            }
            T1[m * H + v] = acc;
        }
    }
    double bv = -INFINITY;
    int bm = 0, bl = 0;
    for (int m = 0; m < M; ++m)
        for (int l = 0; l < M; ++l) {
            double x = x0 + (double)(l - U) / U, s = 0.0;
            for (int v = 0; v < H; ++v) {
                double a = 2.0 * ORC_PI * v * x / n, wv = (v == 0 || v == n / 2) ? 1.0 : 2.0;
                s += wv * creal(T1[m * H + v] * (cos(a) + I * sin(a)));
            }
            if (s > bv) { bv = s; bm = m; bl = l; }
        }
    free(T1);
    *peak = bv;
    *dx = (x0 < n / 2 ? x0 : x0 - n) + (double)(bl - U) / U;
    *dy = (y0 < n / 2 ? y0 : y0 - n) + (double)(bm - U) / U;
}

/* cross-power spectrum X = conj(St) Sp and its surface, then the up-sampled peak */
void orc_pair_upsampled(const cplx *St, const cplx *Sp, int n, int U, double *peak, double *dx, double *dy) {
    long nn = (long)n * n;
    cplx *X = malloc(sizeof(cplx) * nn);
    double *r = malloc(sizeof(double) * nn);
    for (long k = 0; k < nn; ++k) X[k] = conj(St[k]) * Sp[k];
    orc_xcf_surface(St, Sp, n, r);
    orc_peak_upsampled(X, r, n, U, peak, dx, dy);
    free(X);
    free(r);
}

/* the up-sampled surface at one point (y, x) (the definition above), for the pins */
double orc_upsampled_value(const cplx *St, const cplx *Sp, int n, double y, double x) {
    int H = n / 2 + 1;
    double s = 0.0;
    for (int v = 0; v < H; ++v) {
        cplx acc = 0;
        for (int u = 0; u < n; ++u) {
            double fu = u < n / 2 ? u : u - n;
            double a = 2.0 * ORC_PI * (fu * y + v * x) / n;
            acc += conj(St[(long)u * n + v]) * Sp[(long)u * n + v] * (cos(a) + I * sin(a));
        }
        s += ((v == 0 || v == n / 2) ? 1.0 : 2.0) * creal(acc);
    }
    return s;
}

/* Library search (Fig. 1 A-C): for each pattern, the template whose
 * correlation surface has the highest peak (ties -> lowest template index),
 * that peak, and the sub-pixel shift at it.  St: [T, n, n] full spectra,
 * Sp: [P, n, n].  degenerate[p] != 0 marks a pattern with no signal: best = -1,
 * peak = 0, shift = 0.  peaks_all (nullable) receives the [P, T] matrix of
 * per-template peaks.  Patterns run in parallel (one thread per pattern),
 * each exactly as written above. */
void orc_index(const cplx *St, int T, const cplx *Sp, int P, int n,
               const int32_t *degenerate, int32_t *best, double *peak,
               double *shift, double *peaks_all) {
    long nn = (long)n * n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        double *r = malloc(sizeof(double) * nn);
        if (degenerate && degenerate[p]) {
            best[p] = -1; peak[p] = 0.0; shift[2 * p] = shift[2 * p + 1] = 0.0;
            if (peaks_all) for (int t = 0; t < T; ++t) peaks_all[(long)p * T + t] = 0.0;
            free(r);
            continue;
        }
        int bt = -1;
        double bv = 0.0;
        for (int t = 0; t < T; ++t) {
            orc_xcf_surface(St + (long)t * nn, Sp + (long)p * nn, n, r);
            double m = r[0];
            for (long k = 1; k < nn; ++k) if (r[k] > m) m = r[k];
            if (peaks_all) peaks_all[(long)p * T + t] = m;
            if (bt < 0 || m > bv) { bv = m; bt = t; }
        }
        orc_xcf_surface(St + (long)bt * nn, Sp + (long)p * nn, n, r);
        int sy, sx;
        orc_peak(r, n, &peak[p], &sy, &sx, &shift[2 * p], &shift[2 * p + 1]);
        best[p] = bt;
        free(r);
    }
}

/* Per-pattern pattern centres in the search.  The gnomonic ray of pixel
 * (i, j) is (j + .5 - pcx W, pcy H - (i + .5), pcz W) (projection below), so
 * a pattern centre moved by (dx, dy) in (pcx, pcy) gives every ray to the
 * pixel dx W columns right and dy H rows down: the screen content of the
 * pattern is the library-centre projection translated by exactly
 * (dx W, dy H) px.  The search keeps the library's templates, and this takes
 * that translation out of the measured shift, so that what remains is the
 * orientation's part (the refinement section's per-pattern centre).  pcz is
 * a scale, not a translation, and is not corrected.  Degenerate patterns
 * (best < 0) keep their zero shift. */
void orc_pc_shift(const double *pcs, int P, double pcx, double pcy, int W, int H,
                  const int32_t *best, double *shift) {
    for (int p = 0; p < P; ++p) {
        if (best[p] < 0) continue;
        shift[2 * p] -= (pcs[3 * p] - pcx) * W;
        shift[2 * p + 1] -= (pcs[3 * p + 1] - pcy) * H;
    }
}

/* ---------------------------------------------------------------------- */
/* master pattern lookup and gnomonic projection (SO(3) Library Generation) */
/* ---------------------------------------------------------------------- */

/* Rosca (2010) equal-area map of the northern hemisphere onto the square
 * [-sqrt(pi/2), sqrt(pi/2)]^2; the southern hemisphere uses (x, y, -z). */
void orc_lambert_forward(const double v[3], double *X, double *Y) {
    double x = v[0], y = v[1], z = fabs(v[2]);
    double q = sqrt(2.0 * (1.0 - z));
    double sp = sqrt(ORC_PI) / 2.0, ts = 2.0 / sqrt(ORC_PI);
    if (x == 0.0 && y == 0.0) { *X = 0.0; *Y = 0.0; return; }
    if (fabs(y) <= fabs(x)) {
        double s = x >= 0 ? 1.0 : -1.0;
        *X = s * q * sp;
        *Y = s * q * ts * atan(y / x);
    } else {
        double s = y >= 0 ? 1.0 : -1.0;
        *X = s * q * ts * atan(x / y);
        *Y = s * q * sp;
    }
}

/* Inverse of the above (northern hemisphere). */
void orc_lambert_inverse(double X, double Y, double v[3]) {
    if (X == 0.0 && Y == 0.0) { v[0] = 0; v[1] = 0; v[2] = 1; return; }
    if (fabs(Y) <= fabs(X)) {
        double f = (2.0 * X / ORC_PI) * sqrt(ORC_PI - X * X);
        double a = ORC_PI * Y / (4.0 * X);
        v[0] = f * cos(a); v[1] = f * sin(a); v[2] = 1.0 - 2.0 * X * X / ORC_PI;
    } else {
        double f = (2.0 * Y / ORC_PI) * sqrt(ORC_PI - Y * Y);
        double a = ORC_PI * X / (4.0 * Y);
        v[0] = f * sin(a); v[1] = f * cos(a); v[2] = 1.0 - 2.0 * Y * Y / ORC_PI;
    }
}

/* Master intensity in direction v (unit): Lambert square coordinates, then
 * bilinear interpolation between the four nearest cell centres of the
 * hemisphere's M x M grid (cell (a, b) centred at X = L(2(b+.5)/M - 1),
 * Y = L(2(a+.5)/M - 1)), clamped at the square's edge.  master: [2, M, M]. */
/* Keys' cubic convolution weight (a = -1/2), the interpolation kernel of the
 * paper's bicubic reprojection (its exact kernel is not given; reading). */
static double keys_w(double t) {
    t = fabs(t);
    const double a = -0.5;
    if (t <= 1.0) return (a + 2.0) * t * t * t - (a + 3.0) * t * t + 1.0;
    if (t < 2.0) return a * t * t * t - 5.0 * a * t * t + 8.0 * a * t - 4.0 * a;
    return 0.0;
}

/* value of one hemisphere's M x M grid at grid coordinates (fx, fy) (cell
 * centres at integers), clamped to [0, M - 1]; interp 0 bilinear, 1 bicubic
 * (4 x 4 cell centres, indices clamped at the edges) */
double orc_grid_interp(const float *g, int M, double fx, double fy, int interp) {
    if (fx < 0) fx = 0;
    if (fx > M - 1) fx = M - 1;
    if (fy < 0) fy = 0;
    if (fy > M - 1) fy = M - 1;
    if (interp == 1) {
        const int i0 = (int)floor(fx), j0 = (int)floor(fy);
        double s = 0.0;
        for (int dj = -1; dj <= 2; ++dj) {
            int j = j0 + dj;
            j = j < 0 ? 0 : (j > M - 1 ? M - 1 : j);
            const double wy = keys_w(fy - (j0 + dj));
            for (int di = -1; di <= 2; ++di) {
                int i = i0 + di;
                i = i < 0 ? 0 : (i > M - 1 ? M - 1 : i);
                s += wy * keys_w(fx - (i0 + di)) * g[(long)j * M + i];
            }
        }
        return s;
    }
    int i0 = (int)floor(fx), j0 = (int)floor(fy);
    if (i0 > M - 2) i0 = M - 2;
    if (j0 > M - 2) j0 = M - 2;
    double tx = fx - i0, ty = fy - j0;
    double a = g[(long)j0 * M + i0], b = g[(long)j0 * M + i0 + 1];
    double c = g[(long)(j0 + 1) * M + i0], d = g[(long)(j0 + 1) * M + i0 + 1];
    return (1 - ty) * ((1 - tx) * a + tx * b) + ty * ((1 - tx) * c + tx * d);
}

/* master lookup with the chosen interpolation (0 bilinear, 1 bicubic) */
double orc_master_lookup_interp(const float *master, int M, const double v[3], int interp) {
    double X, Y;
    orc_lambert_forward(v, &X, &Y);
    double L = sqrt(ORC_PI / 2.0);
    double fx = (X / L + 1.0) * M / 2.0 - 0.5;
    double fy = (Y / L + 1.0) * M / 2.0 - 0.5;
    return orc_grid_interp(master + (v[2] >= 0.0 ? 0 : (long)M * M), M, fx, fy, interp);
}

double orc_master_lookup(const float *master, int M, const double v[3]) {
    double X, Y;
    orc_lambert_forward(v, &X, &Y);
    double L = sqrt(ORC_PI / 2.0);
    double fx = (X / L + 1.0) * M / 2.0 - 0.5;
    double fy = (Y / L + 1.0) * M / 2.0 - 0.5;
    if (fx < 0) fx = 0;
    if (fx > M - 1) fx = M - 1;
    if (fy < 0) fy = 0;
    if (fy > M - 1) fy = M - 1;
    int i0 = (int)floor(fx), j0 = (int)floor(fy);
    if (i0 > M - 2) i0 = M - 2;
    if (j0 > M - 2) j0 = M - 2;
    double tx = fx - i0, ty = fy - j0;
    const float *g = master + (v[2] >= 0.0 ? 0 : (long)M * M);
    double a = g[(long)j0 * M + i0], b = g[(long)j0 * M + i0 + 1];
    double c = g[(long)(j0 + 1) * M + i0], d = g[(long)(j0 + 1) * M + i0 + 1];
    return (1 - ty) * ((1 - tx) * a + tx * b) + ty * ((1 - tx) * c + tx * d);
}

/* Rotation matrix of unit quaternion (w, x, y, z), row-major. */
void orc_quat_to_matrix(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* Gnomonic projection of the master pattern onto an n x n detector for
 * orientation q (reprojection of the master pattern, SO(3) Library Generation
 * section).  Pixel (i, j) (row from the top, column from the left, centres at
 * +0.5) looks along d = (j + .5 - pcx n, pcy n - (i + .5), pcz n) in the
 * detector frame (x right, y up); the sample frame is reached by a rotation
 * about x by 90 - sample_tilt + detector_tilt degrees, and the crystal frame
 * by R(q).  The paper interpolates bicubically on a stereographic master;
 * reading: bilinear on the equal-area master grid.  pc is the (cropped)
 * pattern centre. */
void orc_project_interp(const float *master, int M, const double q[4], const double pc[3],
                        double sample_tilt_deg, double detector_tilt_deg, int n, double *out, int interp);
void orc_project(const float *master, int M, const double q[4], const double pc[3],
                 double sample_tilt_deg, double detector_tilt_deg, int n, double *out) {
    orc_project_interp(master, M, q, pc, sample_tilt_deg, detector_tilt_deg, n, out, 0);
}

/* the projection with the master interpolation of choice (0 bilinear, 1 bicubic) */
void orc_project_interp(const float *master, int M, const double q[4], const double pc[3],
                        double sample_tilt_deg, double detector_tilt_deg, int n, double *out, int interp) {
    double R[9];
    orc_quat_to_matrix(q, R);
    double al = (90.0 - sample_tilt_deg + detector_tilt_deg) * ORC_PI / 180.0;
    double ca = cos(al), sa = sin(al);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double dx = (j + 0.5) - pc[0] * n;
            double dy = pc[1] * n - (i + 0.5);
            double dz = pc[2] * n;
            double nrm = sqrt(dx * dx + dy * dy + dz * dz);
            dx /= nrm; dy /= nrm; dz /= nrm;
            double s[3] = {dx, ca * dy - sa * dz, sa * dy + ca * dz};
            double c[3] = {R[0] * s[0] + R[1] * s[1] + R[2] * s[2],
                           R[3] * s[0] + R[4] * s[1] + R[5] * s[2],
                           R[6] * s[0] + R[7] * s[1] + R[8] * s[2]};
            out[(long)i * n + j] = orc_master_lookup_interp(master, M, c, interp);
        }
}

/* Many projections, one thread per image. quats [P,4], pcs [P,3]. */
void orc_project_many(const float *master, int M, const double *quats, const double *pcs,
                      int P, double sample_tilt_deg, double detector_tilt_deg, int n,
                      double *out, int interp) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < P; ++p)
        orc_project_interp(master, M, quats + 4L * p, pcs + 3L * p, sample_tilt_deg,
                           detector_tilt_deg, n, out + (long)p * n * n, interp);
}

/* Many pre-processings, one thread per image. imgs [P, n, n]. */
void orc_prep_many(const double *imgs, int P, int n, const orc_opts *o, cplx *S,
                   double *y, int32_t *degenerate) {
    long nn = (long)n * n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < P; ++p)
        degenerate[p] = orc_prep(imgs + p * nn, n, o, S + p * nn, y ? y + p * nn : NULL);
}

/* ---------------------------------------------------------------------- */
/* quaternions, symmetry, disorientation (second "Equation 6")             */
/* ---------------------------------------------------------------------- */
static void qmul(const double a[4], const double b[4], double o[4]) {
    double r[4];
    r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    memcpy(o, r, sizeof r);
}

static void qnormalise(double q[4]) {
    double s = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (q[0] < 0) s = -s;
    for (int i = 0; i < 4; ++i) q[i] /= s;
}

void orc_qmul(const double a[4], const double b[4], double o[4]) { qmul(a, b, o); }

/* The 24 proper rotations of the cubic point group 432 as quaternions. */
void orc_cubic_ops(double ops[24][4]) {
    const double h = 0.5, r = sqrt(0.5);
    int k = 0;
    double id[4] = {1, 0, 0, 0};
    memcpy(ops[k++], id, sizeof id);
    for (int ax = 1; ax <= 3; ++ax) {          /* 180 deg about x, y, z */
        double q[4] = {0, 0, 0, 0}; q[ax] = 1; memcpy(ops[k++], q, sizeof q);
    }
    for (int ax = 1; ax <= 3; ++ax)            /* +-90 deg about x, y, z */
        for (int s = -1; s <= 1; s += 2) {
            double q[4] = {r, 0, 0, 0}; q[ax] = s * r; memcpy(ops[k++], q, sizeof q);
        }
    for (int sx = -1; sx <= 1; sx += 2)        /* +-120 deg about <111> */
        for (int sy = -1; sy <= 1; sy += 2)
            for (int sz = -1; sz <= 1; sz += 2) {
                double q[4] = {h, sx * h, sy * h, sz * h}; memcpy(ops[k++], q, sizeof q);
            }
    const int pairs[3][2] = {{1, 2}, {1, 3}, {2, 3}};  /* 180 deg about <110> */
    for (int p = 0; p < 3; ++p)
        for (int s = -1; s <= 1; s += 2) {
            double q[4] = {0, 0, 0, 0};
            q[pairs[p][0]] = r; q[pairs[p][1]] = s * r;
            memcpy(ops[k++], q, sizeof q);
        }
}

/* Disorientation angle (degrees) between orientations qa and qb of a cubic
 * crystal: the smallest rotation angle of S (qa qb^-1) over the 24 operators
 * S (the paper's minimum over pairs of symmetry operators reduces to one
 * operator because the angle is invariant under conjugation). */
double orc_disorientation(const double qa[4], const double qb[4]) {
    double ops[24][4];
    orc_cubic_ops(ops);
    double binv[4] = {qb[0], -qb[1], -qb[2], -qb[3]};
    double m[4];
    qmul(qa, binv, m);
    double best = 0.0;
    for (int i = 0; i < 24; ++i) {
        double t[4];
        qmul(ops[i], m, t);
        double w = fabs(t[0]) / sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3]);
        if (w > best) best = w;
    }
    if (best > 1.0) best = 1.0;
    return 2.0 * acos(best) * 180.0 / ORC_PI;
}

void orc_disorientation_many(const double *qa, const double *qb, int n, double *out) {
    for (int i = 0; i < n; ++i) out[i] = orc_disorientation(qa + 4L * i, qb + 4L * i);
}

/* ---------------------------------------------------------------------- */
/* refinement (Orientation and Pattern Centre Refinement; Eq. 7, Fig. 6)   */
/* ---------------------------------------------------------------------- */

/* Log-polar resampling of an n x n image about the screen centre
 * c = (n/2 - 0.5, n/2 - 0.5): radii r_m = rmin (rmax/rmin)^(m/(nr-1)),
 * angles eta_l = 2 pi l / neta counter-clockwise from +x (y up), sample at
 * column c + r cos(eta), row c - r sin(eta), bilinear.  The paper centres the
 * transform at the screen centre; the sampling constants are a reading. */
void orc_logpolar(const double *img, int n, int nr, int neta, double rmin, double rmax,
                  double *out) {
    double c = n / 2.0 - 0.5;
    for (int m = 0; m < nr; ++m) {
        double r = rmin * pow(rmax / rmin, nr > 1 ? (double)m / (nr - 1) : 0.0);
        for (int l = 0; l < neta; ++l) {
            double eta = 2.0 * ORC_PI * l / neta;
            double fx = c + r * cos(eta), fy = c - r * sin(eta);
            int x0 = (int)floor(fx), y0 = (int)floor(fy);
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x0 > n - 2) x0 = n - 2;
            if (y0 > n - 2) y0 = n - 2;
            double tx = fx - x0, ty = fy - y0;
            double a = img[(long)y0 * n + x0], b = img[(long)y0 * n + x0 + 1];
            double cc = img[(long)(y0 + 1) * n + x0], d = img[(long)(y0 + 1) * n + x0 + 1];
            out[(long)m * neta + l] = (1 - ty) * ((1 - tx) * a + tx * b) + ty * ((1 - tx) * cc + tx * d);
        }
    }
}

/* Correlation along eta of two log-polar images (rotation about the screen
 * centre becomes a shift along eta): both are made zero-mean, then
 * c(D) = sum_m sum_l a[m][l] b[m][(l + D) mod neta] / (|a| |b|), computed by
 * its definition.  Returns the shift D (argmax, ties -> lowest, wrapped into
 * [-neta/2, neta/2), plus the parabolic offset) and the peak value.  b equal
 * to a rotated counter-clockwise by theta peaks at D = theta neta / 2 pi. */
double orc_eta_xcf(const double *a_in, const double *b_in, int nr, int neta, double *peak,
                   double *c_out) {
    long tot = (long)nr * neta;
    double *a = malloc(sizeof(double) * tot), *b = malloc(sizeof(double) * tot);
    double *c = c_out ? c_out : malloc(sizeof(double) * neta);
    double ma = 0, mb = 0;
    for (long k = 0; k < tot; ++k) { ma += a_in[k]; mb += b_in[k]; }
    ma /= tot; mb /= tot;
    double na = 0, nb = 0;
    for (long k = 0; k < tot; ++k) {
        a[k] = a_in[k] - ma; b[k] = b_in[k] - mb;
        na += a[k] * a[k]; nb += b[k] * b[k];
    }
    double nrm = sqrt(na * nb);
    if (!(nrm > 0)) nrm = 1.0;
    for (int D = 0; D < neta; ++D) {
        double s = 0.0;
        for (int m = 0; m < nr; ++m)
            for (int l = 0; l < neta; ++l)
                s += a[(long)m * neta + l] * b[(long)m * neta + (l + D) % neta];
        c[D] = s / nrm;
    }
    int best = 0;
    for (int D = 1; D < neta; ++D) if (c[D] > c[best]) best = D;
    double off = orc_parabola(c[(best + neta - 1) % neta], c[best], c[(best + 1) % neta]);
    *peak = c[best];
    double sh = (best < neta / 2 ? best : best - neta) + off;
    free(a); free(b);
    if (!c_out) free(c);
    return sh;
}

/* The Z measurement with multiple windows (the refinement section correlates
 * "multiple windows" of the log-polar images and keeps only the shift along
 * eta; reading: W radial bands, band w holding radii [w nr / W, (w+1) nr / W)
 * (integer division), each correlated along eta on its own as orc_eta_xcf
 * does for the whole image, the shift the median of the W band shifts (the
 * mean of the middle two for even W)).  W <= 1 is orc_eta_xcf.  *peak gets
 * the largest band peak. */
double orc_eta_windows(const double *a, const double *b, int nr, int neta, int W, double *peak) {
    if (W <= 1) return orc_eta_xcf(a, b, nr, neta, peak, NULL);
    if (W > nr) W = nr;
    double *sh = malloc(sizeof(double) * W), best = -2.0;
    for (int w = 0; w < W; ++w) {
        int m0 = w * nr / W, m1 = (w + 1) * nr / W;
        double pk;
        sh[w] = orc_eta_xcf(a + (long)m0 * neta, b + (long)m0 * neta, m1 - m0, neta, &pk, NULL);
        if (pk > best) best = pk;
    }
    for (int i = 1; i < W; ++i)   /* insertion sort */
        for (int j = i; j > 0 && sh[j] < sh[j - 1]; --j) {
            double t = sh[j]; sh[j] = sh[j - 1]; sh[j - 1] = t;
        }
    double med = W % 2 ? sh[W / 2] : 0.5 * (sh[W / 2 - 1] + sh[W / 2]);
    free(sh);
    *peak = best;
    return med;
}

/* q_new = q (x) q_s (x) conj(qQ) (x) conj(q_s): the orientation whose template
 * equals the template of q rotated by the detector-frame rotation Q (q_s is
 * the detector -> sample rotation about x). */
static void apply_detector_rotation(const double q[4], const double qQ[4], double al,
                                    double out[4]) {
    double qs[4] = {cos(al / 2), sin(al / 2), 0, 0};
    double qsi[4] = {qs[0], -qs[1], 0, 0};
    double qQi[4] = {qQ[0], -qQ[1], -qQ[2], -qQ[3]};
    double t1[4], t2[4];
    qmul(q, qs, t1);
    qmul(t1, qQi, t2);
    qmul(t2, qsi, out);
    qnormalise(out);
}

/* Refine one pattern from a seed orientation (the refinement section):
 * for each iteration
 *   X/Y: project the template at the current orientation with the pattern's
 *        PC, pre-process, cross-correlate with the pattern -> sub-pixel shift
 *        (dx, dy); a rotation about the detector y (x) axis is a horizontal
 *        (vertical) shift, theta = atan(shift / L), L = pcz n (Eq. 7, with
 *        atan in place of the small-angle ratio); compose;
 *   Z:   re-project at the updated orientation, pre-process, log-polar
 *        transform the filtered spatial images of template and pattern about
 *        the screen centre, correlate along eta -> rotation about the
 *        detector z axis; compose;
 * and stop when the total update of the iteration is below tol_deg or after
 * max_it iterations (the paper finds about two iterations suffice).
 * Returns 0; q_out receives the refined orientation, *peak_out the XCF peak of
 * the last X/Y step, *iters_out the iterations performed, and (nullable)
 * trace[it*4 + 0..3] = (dx, dy, deta, update_deg) of each iteration. */
int orc_refine_one(const float *master, int M, const double pc[3], double sample_tilt_deg,
                   double detector_tilt_deg, const orc_opts *o, const float *pattern, int n,
                   const double q_seed[4], int max_it, double tol_deg, double q_out[4],
                   double *peak_out, int32_t *iters_out, double *trace) {
    long nn = (long)n * n;
    double *img = malloc(sizeof(double) * nn), *yP = malloc(sizeof(double) * nn);
    double *yT = malloc(sizeof(double) * nn), *r = malloc(sizeof(double) * nn);
    cplx *SP = malloc(sizeof(cplx) * nn), *ST = malloc(sizeof(cplx) * nn);
    int nr = o->lp_nr, ne = o->lp_neta;
    double *lpP = malloc(sizeof(double) * nr * ne), *lpT = malloc(sizeof(double) * nr * ne);
    for (long k = 0; k < nn; ++k) img[k] = pattern[k];
    orc_prep(img, n, o, SP, yP);
    orc_logpolar(yP, n, nr, ne, o->lp_rmin, o->lp_rmax, lpP);
    double al = (90.0 - sample_tilt_deg + detector_tilt_deg) * ORC_PI / 180.0;
    double L = pc[2] * n;
    double q[4] = {q_seed[0], q_seed[1], q_seed[2], q_seed[3]};
    qnormalise(q);
    double peak = 0.0;
    int it = 0;
    while (it < max_it) {
        /* X/Y step */
        orc_project_interp(master, M, q, pc, sample_tilt_deg, detector_tilt_deg, n, img, o->interp);
        orc_prep(img, n, o, ST, NULL);
        orc_xcf_surface(ST, SP, n, r);
        int sy, sx;
        double dx, dy;
        if (o->upsample >= 2)
            orc_pair_upsampled(ST, SP, n, o->upsample, &peak, &dx, &dy);
        else
            orc_peak(r, n, &peak, &sy, &sx, &dx, &dy);
        double tx = atan(dy / L), ty = atan(dx / L);
        double qx[4] = {cos(tx / 2), sin(tx / 2), 0, 0};
        double qy[4] = {cos(ty / 2), 0, sin(ty / 2), 0};
        double qQ[4], q1[4];
        qmul(qx, qy, qQ);
        apply_detector_rotation(q, qQ, al, q1);
        /* Z step */
        orc_project_interp(master, M, q1, pc, sample_tilt_deg, detector_tilt_deg, n, img, o->interp);
        orc_prep(img, n, o, ST, yT);
        orc_logpolar(yT, n, nr, ne, o->lp_rmin, o->lp_rmax, lpT);
        double zpk;
        double deta = orc_eta_windows(lpT, lpP, nr, ne, o->lp_windows, &zpk);
        double tz = 2.0 * ORC_PI * deta / ne;
        double qz[4] = {cos(tz / 2), 0, 0, sin(tz / 2)};
        double q2[4];
        apply_detector_rotation(q1, qz, al, q2);
        double dot = fabs(q2[0] * q[0] + q2[1] * q[1] + q2[2] * q[2] + q2[3] * q[3]);
        if (dot > 1.0) dot = 1.0;
        double upd = 2.0 * acos(dot) * 180.0 / ORC_PI;
        if (trace) {
            trace[4 * it + 0] = dx; trace[4 * it + 1] = dy;
            trace[4 * it + 2] = deta; trace[4 * it + 3] = upd;
        }
        memcpy(q, q2, sizeof q);
        ++it;
        if (upd < tol_deg) break;
    }
    memcpy(q_out, q, sizeof q);
    *peak_out = peak;
    *iters_out = it;
    free(img); free(yP); free(yT); free(r); free(SP); free(ST); free(lpP); free(lpT);
    return 0;
}

/* Refine many patterns, one thread per pattern. patterns [P, n, n] (cropped),
 * pcs [P, 3] (cropped PCs), seeds [P, 4]. */
void orc_refine_many(const float *master, int M, const double *pcs, double sample_tilt_deg,
                     double detector_tilt_deg, const orc_opts *o, const float *patterns,
                     int P, int n, const double *seeds, int max_it, double tol_deg,
                     double *quats, double *peaks, int32_t *iters) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p)
        orc_refine_one(master, M, pcs + 3L * p, sample_tilt_deg, detector_tilt_deg, o,
                       patterns + (long)p * n * n, n, seeds + 4L * p, max_it, tol_deg,
                       quats + 4L * p, peaks + p, iters + p, NULL);
}

/* ---------------------------------------------------------------------- */
/* zero-shift screen (Eq. 1: the normalised dot product is the correlation  */
/* at zero shift of the unit-norm filtered images)                         */
/* ---------------------------------------------------------------------- */

/* Round to the nearest BF16 value (ties to even) through float32, the
 * rounding the tensor-core operands receive. */
double orc_bf16_round(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* S[p][t] = sum_k yp[p][k] yt[t][k] in FP64; with bf16 != 0 every input is
 * first rounded to BF16 (so that only the accumulation differs from the
 * tensor cores).  yp [P][K], yt [T][K]. */
void orc_screen(const double *yp, int P, const double *yt, int T, long K, int bf16, double *S) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p)
        for (int t = 0; t < T; ++t) {
            double s = 0.0;
            for (long k = 0; k < K; ++k) {
                double a = yp[(long)p * K + k], b = yt[(long)t * K + k];
                if (bf16) { a = orc_bf16_round(a); b = orc_bf16_round(b); }
                s += a * b;
            }
            S[(long)p * T + t] = s;
        }
}

/* ---------------------------------------------------------------------- */
/* normalised dot product (Eq. 1) and the peak-width experiments of the     */
/* sampling-frequency section (Figs. 3 and 4)                              */
/* ---------------------------------------------------------------------- */

/* Contrast normalisation of the NDP (NDP section; the simulation set-up of
 * the sampling-frequency section): zero mean and unit population standard
 * deviation over the d pixels.  Returns 1 and zeros for a constant image (the
 * same degeneracy test as orc_prep). */
int orc_ndp_normalise(const double *img, long d, double *out) {
    double mean = 0.0;
    for (long i = 0; i < d; ++i) mean += img[i];
    mean /= d;
    double var = 0.0;
    for (long i = 0; i < d; ++i) var += (img[i] - mean) * (img[i] - mean);
    var /= d;
    double sd = sqrt(var);
    if (!(sd > 1e-12 * (1.0 + fabs(mean)))) {
        memset(out, 0, sizeof(double) * d);
        return 1;
    }
    for (long i = 0; i < d; ++i) out[i] = (img[i] - mean) / sd;
    return 0;
}

/* Background correction before the NDP (the NDP section and the simulation
 * set-up of the sampling-frequency section correct the background of every
 * pattern and template first, drawing out the bands; the paper names the
 * routine but not its form).  Reading: subtract the Gaussian-blurred image,
 * blur = separable Gaussian of standard deviation sigma pixels with weights
 * exp(-k^2 / (2 sigma^2)), k = -R..R, R = floor(3 sigma + 1/2), normalised to
 * sum 1, and edge pixels repeated beyond the border.  sigma = 0 takes n / 8
 * (the value that indexed the synthetic noisy maps best); sigma < 0 copies
 * the image unchanged.  img, out [n][n]. */
void orc_ndp_background(const double *img, int n, double sigma, double *out) {
    long nn = (long)n * n;
    if (sigma < 0) {
        memcpy(out, img, sizeof(double) * nn);
        return;
    }
    if (sigma == 0) sigma = n / 8.0;
    int R = (int)(3.0 * sigma + 0.5);
    double *w = malloc(sizeof(double) * (2 * R + 1)), sw = 0.0;
    for (int k = -R; k <= R; ++k) sw += (w[k + R] = exp(-(double)k * k / (2.0 * sigma * sigma)));
    for (int k = 0; k <= 2 * R; ++k) w[k] /= sw;
    double *rows = malloc(sizeof(double) * nn);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = -R; k <= R; ++k) {
                int c = j + k < 0 ? 0 : (j + k >= n ? n - 1 : j + k);
                s += w[k + R] * img[(long)i * n + c];
            }
            rows[(long)i * n + j] = s;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = -R; k <= R; ++k) {
                int r = i + k < 0 ? 0 : (i + k >= n ? n - 1 : i + k);
                s += w[k + R] * rows[(long)r * n + j];
            }
            out[(long)i * n + j] = img[(long)i * n + j] - s;
        }
    free(w); free(rows);
}

/* Eq. 1 for one pair: the mean over the d pixels of the products of the two
 * contrast-normalised images.  Reading: the printed formula carries both a
 * 1/d and the two vector norms, which would give 1/d for identical images,
 * while the text fixes that value at 1; with unit-variance images the norms
 * are sqrt(d) and one normalisation is kept, making the NDP the cosine of the
 * angle between the mean-removed pixel vectors.  0 if either image is
 * constant. */
double orc_ndp(const double *a, const double *b, long d) {
    double *na = malloc(sizeof(double) * d), *nb = malloc(sizeof(double) * d);
    int da = orc_ndp_normalise(a, d, na), db = orc_ndp_normalise(b, d, nb);
    double s = 0.0;
    if (!da && !db)
        for (long i = 0; i < d; ++i) s += na[i] * nb[i];
    free(na); free(nb);
    return s / d;
}

/* Dictionary indexing with Eq. 1 (the NDP section): for each pattern the
 * template of largest NDP (ties -> lowest index) and that NDP; scores
 * (nullable) receives all P x T values.  pats [P][d], tmpl [T][d]; a constant
 * pattern gets best = -1 and score 0. */
void orc_ndp_index(const double *pats, int P, const double *tmpl, int T, long d, int32_t *best,
                   double *score, double *scores) {
    double *nt = malloc(sizeof(double) * d * T);
    for (int t = 0; t < T; ++t) orc_ndp_normalise(tmpl + (long)t * d, d, nt + (long)t * d);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        double *np_ = malloc(sizeof(double) * d);
        int deg = orc_ndp_normalise(pats + (long)p * d, d, np_);
        int b = -1;
        double bs = 0.0;
        for (int t = 0; t < T; ++t) {
            double s = 0.0;
            for (long i = 0; i < d; ++i) s += np_[i] * nt[(long)t * d + i];
            s /= d;
            if (scores) scores[(long)p * T + t] = s;
            if (!deg && (b < 0 || s > bs)) { b = t; bs = s; }
        }
        best[p] = b;
        score[p] = deg ? 0.0 : bs;
        free(np_);
    }
    free(nt);
}

/* Test orientation of the rotation experiment (sampling-frequency section):
 * the crystal of q rotated by theta (radians) about axis `axis` (0 x, 1 y,
 * 2 z) of the detector frame, i.e. the orientation whose pattern is the
 * pattern of q rotated by that detector-frame rotation (the composition the
 * refinement applies). */
void orc_scan_orientation(const double q[4], int axis, double theta, double sample_tilt_deg,
                          double detector_tilt_deg, double out[4]) {
    double al = (90.0 - sample_tilt_deg + detector_tilt_deg) * ORC_PI / 180.0;
    double qQ[4] = {cos(theta / 2), 0, 0, 0};
    qQ[1 + axis] = sin(theta / 2);
    apply_detector_rotation(q, qQ, al, out);
}

/* The rotation experiment of Fig. 3: a reference pattern of orientation q at
 * pattern centre pc_ref against test patterns rotated about the detector x, y
 * and z axes by theta_j = (j - nh) step_deg, j = 0..2 nh, projected at pc_test
 * (the PC-error experiment of Fig. 4 A-C when pc_test differs).  For each
 * axis a and step j:
 *   ndp[a L + j] = Eq. 1 between reference and test (background-corrected,
 *                  contrast-normalised);
 *   xcf[a L + j] = peak of the FFT cross-correlation (Eqs. 4-6: window,
 *                  band-pass, unit-norm spectra; integer peak, or the
 *                  up-sampled peak when o->upsample >= 2), reference as the
 *                  template, 0 if either image is degenerate;
 * L = 2 nh + 1.  pcs are those of the n x n (cropped) screen.  The NDP
 * compares the background-corrected images (orc_ndp_background with
 * o->ndp_bg_sigma), the FFT the raw ones through its own filters. */
void orc_rotation_scan(const float *master, int M, int n, const double pc_ref[3], const double pc_test[3],
                       double sample_tilt_deg, double detector_tilt_deg, const orc_opts *o,
                       const double q[4], int nh, double step_deg, double *ndp, double *xcf) {
    long nn = (long)n * n;
    int L = 2 * nh + 1;
    double *ref = malloc(sizeof(double) * nn), *refb = malloc(sizeof(double) * nn);
    cplx *Sr = malloc(sizeof(cplx) * nn);
    orc_project_interp(master, M, q, pc_ref, sample_tilt_deg, detector_tilt_deg, n, ref, o->interp);
    orc_ndp_background(ref, n, o->ndp_bg_sigma, refb);
    int dref = orc_prep(ref, n, o, Sr, NULL);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < 3 * L; ++k) {
        int a = k / L, j = k % L;
        double qt[4];
        orc_scan_orientation(q, a, (j - nh) * step_deg * ORC_PI / 180.0, sample_tilt_deg,
                             detector_tilt_deg, qt);
        double *img = malloc(sizeof(double) * nn), *r = malloc(sizeof(double) * nn);
        cplx *St = malloc(sizeof(cplx) * nn);
        orc_project_interp(master, M, qt, pc_test, sample_tilt_deg, detector_tilt_deg, n, img, o->interp);
        orc_ndp_background(img, n, o->ndp_bg_sigma, r);
        ndp[k] = orc_ndp(refb, r, nn);
        int dt = orc_prep(img, n, o, St, NULL);
        double pk = 0.0;
        if (!dref && !dt) {
            if (o->upsample >= 2) {
                double dx, dy;
                orc_pair_upsampled(Sr, St, n, o->upsample, &pk, &dx, &dy);
            } else {
                int sy, sx;
                double dx, dy;
                orc_xcf_surface(Sr, St, n, r);
                orc_peak(r, n, &pk, &sy, &sx, &dx, &dy);
            }
        }
        xcf[k] = pk;
        free(img); free(r); free(St);
    }
    free(ref); free(refb); free(Sr);
}

/* Full width at half maximum of a correlation-versus-angle curve (the
 * sampling-frequency section measures the peak width of Fig. 3 this way):
 * c[j] sampled at theta_j = (j - (L - 1) / 2) step, the maximum at the lowest
 * index of the largest value, half = max / 2 (the maximum's half height over
 * zero correlation); walking outwards from the maximum to the first sample
 * below half on each side, each crossing is placed by linear interpolation
 * between that sample and its inner neighbour.  Returns the width (units of
 * step), or -1 when the curve does not fall below half on both sides within
 * the scan or its maximum is not positive. */
double orc_fwhm(const double *c, int L, double step) {
    int m = 0;
    for (int j = 1; j < L; ++j)
        if (c[j] > c[m]) m = j;
    if (!(c[m] > 0.0)) return -1.0;
    double h = 0.5 * c[m];
    int l = m, r = m;
    while (l > 0 && c[l - 1] >= h) --l;
    while (r < L - 1 && c[r + 1] >= h) ++r;
    if (l == 0 || r == L - 1) return -1.0;
    double tl = (l - 1) + (h - c[l - 1]) / (c[l] - c[l - 1]);
    double tr = r + (c[r] - h) / (c[r] - c[r + 1]);
    return (tr - tl) * step;
}

/* ---------------------------------------------------------------------- */
/* SO(3) sampling: the library generator and the nearest-neighbour study   */
/* (SO(3) Library Generation, Sampling Frequency; Eq. 6 (the second); Fig. 2) */
/* ---------------------------------------------------------------------- */

/* Bunge (phi1, Phi, phi2) -> q = qz(phi1) qx(Phi) qz(phi2), unit, w >= 0. */
static void bunge_to_quat(double p1, double P, double p2, double q[4]) {
    double a[4] = {cos(p1 / 2), 0, 0, sin(p1 / 2)}, b[4] = {cos(P / 2), sin(P / 2), 0, 0};
    double c[4] = {cos(p2 / 2), 0, 0, sin(p2 / 2)}, t[4];
    qmul(a, b, t);
    qmul(t, c, q);
    qnormalise(q);
    if (q[0] < 0) for (int i = 0; i < 4; ++i) q[i] = -q[i];
}

/* Cubic (432) fundamental zone in Rodrigues space: |r_i| <= sqrt(2) - 1 and
 * |r_1| + |r_2| + |r_3| <= 1, r = (x, y, z) / w; faces included (1e-12). */
static int in_cubic_fz(const double q[4]) {
    double w = q[0] > 1e-300 ? q[0] : 1e-300;
    double r0 = fabs(q[1]) / w, r1 = fabs(q[2]) / w, r2 = fabs(q[3]) / w;
    double m = r0 > r1 ? (r0 > r2 ? r0 : r2) : (r1 > r2 ? r1 : r2);
    return m <= sqrt(2.0) - 1.0 + 1e-12 && r0 + r1 + r2 <= 1.0 + 1e-12;
}

/* The library generator (SO(3) Library Generation section: MTEX's S^2 x S^1
 * scheme): the polar angle of S^2 split into n_p = round(pi / d) equal steps,
 * ring i sampled at n_a = max(1, round(2 pi sin(Phi_i) / d)) azimuths (offset
 * by half a step on odd rings), the rotation about each S^2 point (S^1) split
 * into n_s = round(2 pi / d) equal steps; orientation = Bunge (azimuth, Phi,
 * S^1 angle); kept where it falls in the cubic fundamental zone, in
 * generation order (ring, azimuth, S^1).  Reading: points on the zone's faces
 * are kept, and with dedup != 0 a point whose disorientation to an earlier
 * in-zone grid point is below 1e-3 deg (a symmetry copy across a face) is
 * dropped.
 * Rounding: halves away from zero.  Writes at most cap orientations [cap][4]
 * (out may be NULL) and returns the count. */
long orc_so3_grid(double step_deg, int dedup, double *out, long cap) {
    double d = step_deg * ORC_PI / 180.0;
    long np_ = lround(ORC_PI / d), ns = lround(2 * ORC_PI / d);
    if (np_ < 1) np_ = 1;
    if (ns < 1) ns = 1;
    long n = 0, nc = 0, cand_cap = 1024;
    double *cand = malloc(sizeof(double) * 4 * cand_cap);   /* every in-zone point so far */
    for (long i = 0; i <= np_; ++i) {
        double Phi = ORC_PI * i / np_;
        long na = lround(2 * ORC_PI * sin(Phi) / d);
        if (na < 1) na = 1;
        for (long j = 0; j < na; ++j) {
            double p1 = 2 * ORC_PI * (j + 0.5 * (i % 2)) / na;
            for (long k = 0; k < ns; ++k) {
                double q[4];
                bunge_to_quat(p1, Phi, 2 * ORC_PI * k / ns, q);
                if (!in_cubic_fz(q)) continue;
                int dup = 0;
                for (long m = 0; dedup && m < nc && !dup; ++m)
                    dup = orc_disorientation(q, cand + 4 * m) < 1e-3;
                if (nc == cand_cap) {
                    cand_cap *= 2;
                    cand = realloc(cand, sizeof(double) * 4 * cand_cap);
                }
                memcpy(cand + 4 * nc++, q, sizeof q);
                if (dup) continue;
                if (out && n < cap) memcpy(out + 4 * n, q, sizeof q);
                ++n;
            }
        }
    }
    free(cand);
    return n;
}

/* Nearest neighbour under the cubic disorientation (the Fig. 2 study measures
 * every library orientation's disorientation to its closest other member):
 * for each qa[i], the qb[j] of smallest disorientation (ties -> lowest j) over
 * j != i (mode 1: the two sets are one), j < i (mode 2), or every j (mode 0);
 * angle in degrees, -1 and index -1 when there is no candidate. */
void orc_nearest_disorientation(const double *qa, int na, const double *qb, int nb, int mode,
                                double *angle, int32_t *index) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < na; ++i) {
        double best = -1.0;
        int bj = -1;
        int lim = mode == 2 ? (i < nb ? i : nb) : nb;
        for (int j = 0; j < lim; ++j) {
            if (mode == 1 && j == i) continue;
            double a = orc_disorientation(qa + 4L * i, qb + 4L * j);
            if (bj < 0 || a < best) { best = a; bj = j; }
        }
        angle[i] = best;
        index[i] = bj;
    }
}
