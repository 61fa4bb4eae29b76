/*
 * ebsdxcf — GB300 (sm_103a) EBSD pattern indexing by FFT cross-correlation
 * template matching with orientation refinement, after Foden, Collins,
 * Wilkinson & Britton, "Indexing Electron Backscatter Diffraction Patterns
 * with a Refined Template Matching Approach" (arXiv 1807.11313).
 *
 * C ABI.  Conventions for every entry point:
 *  - Return value: XCF_OK (0) or a negative XCF_ERR_* code; nothing throws
 *    across the ABI.  xcf_strerror() names a code, xcf_last_error() gives the
 *    detail of the last failing call on a context.
 *  - Array arguments are DEVICE pointers owned by the caller, row-major and
 *    contiguous, unless the entry point's name ends in _host (then they are
 *    host pointers, ideally pinned).  Struct arguments (options, geometry) are
 *    host pointers read during the call.
 *  - Work is enqueued on the caller's `stream` (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and is asynchronous unless stated.
 *  - A context owns reusable device scratch.  One context must not be used
 *    from two host threads or on two streams at once.
 *  - Geometry: a W x H detector, pixel (i, j) = (row from the top, column from
 *    the left); Bruker-style pattern centre (pcx of the width from the left,
 *    pcy of the height from the top, detector distance pcz x width).  The
 *    indexer works on the centred square crop of side N = the largest power
 *    of two <= min(W, H) (capped at 256, at least 16), with the PC moved so
 *    that it still points at the same pixel (paper, FFT section, footnotes 1-2).
 *  - Orientations are unit quaternions (w, x, y, z) in float64; R(q) maps
 *    sample-frame directions to crystal-frame directions.
 *  - Spectra are half spectra [N][N/2 + 1] of interleaved float32 (re, im).
 */
#ifndef EBSDXCF_H
#define EBSDXCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XCF_OK                 0
#define XCF_ERR_ARG           -1  /* null pointer, negative count, bad option  */
#define XCF_ERR_SIZE          -2  /* detector below 16 px, or a count too large */
#define XCF_ERR_OOM           -3  /* device allocation failed                  */
#define XCF_ERR_CUDA          -4  /* a CUDA runtime call or launch failed      */
#define XCF_ERR_TIMEOUT       -5  /* a bounded device wait gave up             */
#define XCF_ERR_UNIMPLEMENTED -6  /* combination not built (e.g. NDP at 96 px) */

typedef struct xcf_ctx xcf_ctx;
typedef struct xcf_library xcf_library;

/* Pre-processing and refinement options.  Values <= 0 in the fields marked
 * "auto" take the default for the detector side N. */
typedef struct {
    int32_t window;     /* 0 none, 1 periodic Hann (default)                       */
    double sigma_hp;    /* Gaussian high-pass sigma, cycles/image (default 2)       */
    double sigma_lp;    /* Gaussian low-pass sigma, cycles/image (auto: N/4)        */
    int32_t lp_nr;      /* log-polar radii (auto: N/4)                              */
    int32_t lp_neta;    /* log-polar angles, a power of two (auto: 2N rounded up)   */
    double lp_rmin;     /* smallest log-polar radius, px (auto: N/4)                */
    double lp_rmax;     /* largest log-polar radius, px (auto: N/2 - 1)             */
    int32_t max_iter;   /* refinement iterations (default 2, as in the paper)       */
    double tol_deg;     /* stop when an iteration's update is below this (1e-3)     */
    int32_t upsample;   /* sub-pixel peak: 0 = 3-point parabola per axis (default);
                           U in [2, 20] = the correlation's Fourier series evaluated
                           on a +-1 px grid of step 1/U around the integer peak (the
                           paper's peak "up-sampling"); applies to every peak step
                           (xcf_index shifts and the refinement's X/Y shifts)       */
    int32_t master_interp; /* master-pattern lookup of every projection: 0 = bilinear
                              on the equal-area grid (default); 1 = bicubic (Keys'
                              cubic convolution, a = -1/2), the paper's bicubic
                              reprojection on the same grid                         */
    double ndp_bg_sigma; /* background correction of the NDP (xcf_index_ndp, the NDP
                            curves of xcf_rotation_scan): each crop minus its
                            Gaussian blur of this sigma in px (truncated at
                            round(3 sigma), edges repeated); 0 = N/8 (default),
                            < 0 = no correction                                     */
    int32_t lp_windows;  /* Z step: the log-polar radii split into this many radial
                            windows (at most 16 and lp_nr), each correlated along eta
                            on its own, the rotation the median window shift (the
                            paper's "multiple windows"); 0 = 4 (default), 1 = the
                            whole image as one window                               */
    int32_t native_sizes; /* crop rule: 0 = the largest 2^k square (default, the
                             paper's practice); 1 = the largest of 16, 32, 64, 96,
                             128, 160, 200, 256 px, so that 96, 160 and 200 px
                             detectors are used whole (mixed-radix 3 x 32 and
                             5 x 32 transforms; 8 x 5 x 5 at 200);
                             a library keeps the rule of the context that built it.
                             The NDP calls and the proposal network need 2^k sides */
} xcf_options;

/* Detector geometry of a map (or of a library). */
typedef struct {
    int32_t width, height;      /* detector pixels W, H                         */
    double pcx, pcy, pcz;       /* Bruker-style pattern centre                  */
    double sample_tilt_deg;     /* 70 in the paper                              */
    double detector_tilt_deg;   /* 0                                            */
} xcf_geometry;

/* Text of a status code (static storage). */
const char *xcf_strerror(int code);

/* Detail of the last error on ctx (empty string if none); valid until the
 * next call on ctx. */
const char *xcf_last_error(const xcf_ctx *ctx);

/* Fill *opt with the defaults (paper readings: Hann window, Gaussian
 * band-pass sigma_hp = 2, sigma_lp = N/4; two refinement iterations). */
int xcf_options_default(xcf_options *opt);

/* Square crop rule (paper, FFT section, footnotes 1-2): side n, offsets of the
 * crop in the detector and the pattern centre of the cropped square.  Host
 * only; XCF_ERR_SIZE if the side would be below 16. */
int xcf_crop(const xcf_geometry *g, int32_t *n, int32_t *off_x, int32_t *off_y,
             double pc_out[3]);

/* The same with the crop rule chosen: native = 0 is xcf_crop's 2^k rule, 1 the
 * native rule of xcf_options.native_sizes (the largest of 16, 32, 64, 96, 128,
 * 160, 200, 256 px that fits).  A caller sizing xcf_prep's outputs on a context
 * with native_sizes = 1 takes n from here.  XCF_ERR_ARG if native is not 0/1. */
int xcf_crop_ex(const xcf_geometry *g, int32_t native, int32_t *n, int32_t *off_x,
                int32_t *off_y, double pc_out[3]);

/* Create a context on CUDA device `device` (the device is made current for
 * the call).  opt may be NULL (defaults).  Allocates nothing yet. */
int xcf_create(xcf_ctx **out, const xcf_options *opt, int device);
int xcf_destroy(xcf_ctx *ctx);

/* Gnomonic reprojection of a master pattern onto the detector (paper,
 * "SO(3) Library Generation"): for each of P orientations, pixel (i, j) looks
 * along d = (j + .5 - pcx W, pcy H - (i + .5), pcz W) in the detector frame
 * (x right, y up), is rotated to the sample frame about x by
 * 90 - sample_tilt + detector_tilt degrees and to the crystal frame by R(q),
 * and samples the master bilinearly on its Rosca equal-area square grid.
 *   master  [2, M, M] float32: hemispheres z >= 0 and z < 0; cell (a, b)
 *           centred at X = L(2(b + .5)/M - 1), Y = L(2(a + .5)/M - 1),
 *           L = sqrt(pi/2).
 *   quats   [P, 4] float64.
 *   pcs     [P, 3] float64 per-image pattern centres, or NULL (use g's).
 *   out     [P, H, W] float32.                                              */
int xcf_project(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t P,
                const xcf_geometry *g, const double *pcs, float *out, void *stream);

/* Pre-processing of P detector images (paper, FFT section and the
 * simulation set-up of "SO(3) Sampling Frequency"): centred 2^n crop, zero
 * mean / unit standard deviation, window, 2-D FFT (Eq. 4), band-pass, and
 * division by the filtered spectrum's norm.
 *   images   [P, H, W] float32 (H, W from g).
 *   spectra  [P, N, N/2 + 1, 2] float32 (unit-norm half spectra).
 *   spatial  [P, N, N] float32 or NULL: filtered image = unitary inverse
 *            transform of the unit-norm spectrum (unit L2 norm).
 *   degenerate [P] int32 or NULL: 1 where the image has no signal (zero
 *            variance or no energy in the pass band); its outputs are 0.     */
int xcf_prep(xcf_ctx *ctx, const float *images, int32_t P, const xcf_geometry *g,
             float *spectra, float *spatial, int32_t *degenerate, void *stream);

/* Build a template library (paper, "SO(3) Library Generation"): project the
 * master at each of T orientations on the cropped detector of g, pre-process
 * (as xcf_prep), and keep the half spectra on the device.  The library keeps
 * device copies of the master and of quats (used by refinement).  Input
 * pointers are device pointers and need not outlive the call.  Synchronous
 * with respect to `stream`. */
int xcf_build_library(xcf_ctx *ctx, const float *master, int32_t M, const double *quats,
                      int32_t T, const xcf_geometry *g, xcf_library **out, void *stream);
int xcf_library_free(xcf_library *lib);

/* Build a library from template images the caller simulated elsewhere
 * (images [T, H, W] float32 on g's detector, pre-processed as xcf_prep)
 * with their orientations quats [T, 4]; master [2, M, M] (M >= 2) is kept for
 * refinement and may be NULL (M = 0), in which case xcf_refine fails with
 * XCF_ERR_ARG.  Synchronous with respect to `stream`. */
int xcf_build_library_images(xcf_ctx *ctx, const float *images, const double *quats, int32_t T,
                             const xcf_geometry *g, const float *master, int32_t M,
                             xcf_library **out, void *stream);

/* Library size T, detector side N, and the device pointer to its spectra
 * [T, N, N/2 + 1, 2] (owned by the library; read-only). */
int xcf_library_info(const xcf_library *lib, int32_t *T, int32_t *N, const float **spectra);

/* Library search (paper, Fig. 1 A-C, Eqs. 3 and 6): for each pattern, the
 * template maximising the peak of the normalised cross-correlation surface
 * r(s) = sum_k conj(S_t[k]) S_p[k] exp(+2 pi i k.s / N) over all N^2 circular
 * shifts; ties go to the lowest template index and, within a surface, to the
 * lowest row-major shift.
 *   patterns [P, H, W] float32 with the library's detector (W x H, tilts).
 *   pcs      [P, 3] float64 per-pattern pattern centres (pcx, pcy, pcz), or
 *            NULL (every pattern at the library's centre).  The per-pattern
 *            geometry of a map whose pattern centre drifts across the scan
 *            (paper, refinement section and the large Si map): the templates
 *            stay at the library's centre (the correlation tolerates the
 *            drift as a translation), and the shift is reported relative to
 *            where the template would sit at the pattern's own centre.
 *   best     [P] int32: template index, or -1 for a degenerate pattern.
 *   peak     [P] float32: r at the integer peak of the best template.
 *   shift    [P, 2] float32 (dx, dy) px: the pattern is the template
 *            translated by +shift; integer peak wrapped into [-N/2, N/2) plus a
 *            3-point parabolic sub-pixel offset per axis (the paper's peak
 *            up-sampling, read as a parabola fit), clamped to +-0.5.  With
 *            pcs, minus the translation (pcx_p - pcx_lib) W, (pcy_p - pcy_lib) H
 *            that moving the pattern centre alone produces (a change of pcx
 *            or pcy translates the gnomonic screen content exactly; pcz
 *            scales it and is not corrected).                              */
int xcf_index(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
              const double *pcs, int32_t *best, float *peak, float *shift, void *stream);

/* The same search, but returning every per-template peak: peaks [P, T]
 * float32 (max over shifts of r for each pair).  For analysis and tests. */
int xcf_correlate_all(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                      float *peaks, void *stream);

/* Orientation refinement (paper, "Orientation and Pattern Centre
 * Refinement", Eq. 7, Fig. 6): starting from seeds, each iteration
 *  (X/Y) projects the template at the current orientation with the
 *        pattern's PC, cross-correlates it with the pattern, and turns the
 *        sub-pixel shift (dx, dy) into rotations about the detector y and x
 *        axes, theta = atan(shift / L), L = pcz W (Eq. 7 with atan);
 *  (Z)   re-projects, log-polar transforms the filtered template and pattern
 *        about the screen centre, correlates along the angle and turns the
 *        angular shift into a rotation about the detector z axis;
 * composing each rotation onto the orientation in float64, until the update
 * of an iteration is below tol_deg or max_iter iterations ran.
 *   patterns [P, H, W] float32; seeds [P, 4] float64; pcs [P, 3] float64 or
 *   NULL (library PC): the per-pattern geometry, used by every projection;
 *   max_iter in [1, 1000], or <= 0 for the context's opt.max_iter; tol_deg
 *   >= 0, or < 0 for opt.tol_deg; quats [P, 4] float64 out; peak [P] float32
 *   out (XCF peak of the last X/Y step); iters [P] int32 out.
 * XCF_ERR_ARG if max_iter > 1000.                                          */
int xcf_refine(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
               const double *seeds, const double *pcs, int32_t max_iter, double tol_deg,
               double *quats, float *peak, int32_t *iters, void *stream);

/* Cubic (432) disorientation in degrees between qa[i] and qb[i] (paper, second
 * "Equation 6"): the smallest rotation angle of S qa qb^-1 over the 24 proper
 * cubic operators S.  qa, qb [n, 4] float64; out [n] float64. */
int xcf_disorientation(xcf_ctx *ctx, const double *qa, const double *qb, int32_t n, double *out,
                       void *stream);

/* Library builder with options.  Templates are projected from the master
 * (images == NULL) or pre-processed from the caller's images [T, H, W]
 * (master may then be NULL); flags:
 *   XCF_LIB_SCREEN  also keep each template's unit-norm filtered spatial image
 *                   in BF16 [T, N*N], needed by xcf_screen_topk.
 * Synchronous with respect to `stream`. */
#define XCF_LIB_SCREEN 1
/*   XCF_LIB_NDP     also keep each template's contrast-normalised image (zero
 *                   mean, unit standard deviation over the N x N crop, scaled
 *                   by 1/N so that a plain dot product is Eq. 1) in FP32 and in
 *                   BF16 [T, N*N] each, needed by xcf_index_ndp.              */
#define XCF_LIB_NDP 2
/*   XCF_LIB_NO_SPECTRA  skip the FFT spectra: the library then serves only
 *                   xcf_index_ndp, xcf_screen_topk (with XCF_LIB_SCREEN) and
 *                   the refinement calls; the correlation searches reject it
 *                   with XCF_ERR_ARG.                                         */
#define XCF_LIB_NO_SPECTRA 4
int xcf_build_library_ex(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t T,
                         const xcf_geometry *g, const float *images, int32_t flags, xcf_library **out,
                         void *stream);

/* Zero-shift correlation screen (paper, Eq. 1: the normalised dot product is
 * the correlation at zero shift of the unit-norm filtered images; Eq. 3 is its
 * generalisation to all shifts): score[p, t] = <y_p, y_t> computed on the
 * tensor cores with BF16 operands and FP32 accumulation, and for each pattern
 * the k best templates (1 <= k <= 64) by (score desc, index asc).
 *   cand [P, k] int32 template indices (-1 where T < k); score [P, k] float32.
 * The library must be built with XCF_LIB_SCREEN and hold at most 51,200
 * templates.  Synchronous (it checks the kernel's status word);
 * XCF_ERR_TIMEOUT if a bounded device wait gave up. */
int xcf_screen_topk(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, int32_t k,
                    int32_t *cand, float *score, void *stream);

/* FP32 FFT cross-correlation of each pattern against its own candidate list
 * cand [P, k] (library indices; entries < 0 are skipped) -- the rescore of the
 * precision form.  Outputs as xcf_index (best is a library index). */
int xcf_rescore(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const int32_t *cand,
                int32_t k, int32_t *best, float *peak, float *shift, void *stream);

/* Precision form in one call: per chunk of patterns ONE pre-processing (half
 * spectra and filtered spatial images) serves the BF16 tensor-core screen
 * (top-k by zero-shift score, as xcf_screen_topk), the FP32 XCF rescore of
 * the k candidates (best [P], as xcf_rescore) and the refinement seeded by
 * the best candidate's library orientation (quats [P, 4], peak [P], iters [P],
 * as xcf_refine_best).  The outputs equal the three calls in sequence.  The
 * library needs XCF_LIB_SCREEN and its master pattern; 1 <= k <= 64.  Waits
 * for the device at the end (reports XCF_ERR_TIMEOUT from the screen). */
int xcf_index_precision(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                        const double *pcs, int32_t k, int32_t *best, double *quats, float *peak, int32_t *iters,
                        void *stream);

/* Refinement seeded by library templates: seeds = library orientations of
 * best [P] (identity where best < 0), then xcf_refine. */
int xcf_refine_best(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const int32_t *best,
                    const double *pcs, double *quats, float *peak, int32_t *iters, void *stream);

/* Dictionary indexing with the normalised dot product (paper, Eq. 1 and the
 * NDP section): each pattern's N x N crop is contrast-normalised (zero mean,
 * unit population standard deviation; a constant crop is degenerate), the NDP
 * against every template is computed on the tensor cores with BF16 operands
 * and FP32 accumulation, the k best templates (1 <= k <= 64; score desc,
 * index asc) are rescored in FP32, and the best of those is returned:
 *   best [P] int32 out (-1 for a degenerate pattern), ndp [P] float32 out (its
 *   FP32 NDP, 0 when degenerate); cand [P, k] int32 and cand_score [P, k]
 *   float32 (nullable, together) receive the candidates and their BF16 scores.
 * There is no translation freedom (the NDP compares fixed templates).  The
 * library needs XCF_LIB_NDP and at most 51,200 templates.  Refinement from the
 * result: xcf_refine_best.  Synchronous (XCF_ERR_TIMEOUT if a bounded device
 * wait of the tensor-core pipeline gave up). */
int xcf_index_ndp(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, int32_t k,
                  int32_t *best, float *ndp, int32_t *cand, float *cand_score, void *stream);

/* The peak-width experiment of the sampling-frequency section (Figs. 3 and
 * 4): a reference pattern of orientation q [4] (float64, device) at the
 * geometry's PC, against test patterns of the crystal rotated about the
 * detector x, y and z axes by theta_j = (j - h) step_deg, j = 0 .. 2h,
 * projected at pc_test [3] (detector-frame PC, device; NULL = the geometry's;
 * a different PC is the PC-error experiment of Fig. 4 A-C).  All images are
 * the N x N crop of the detector.  Per axis a and step j:
 *   ndp [3, 2h+1] float32: Eq. 1 between reference and test pattern;
 *   xcf [3, 2h+1] float32: peak of their FFT cross-correlation with the
 *     context's pre-processing (Eqs. 4-6; up-sampled when the option is set),
 *     the reference taken as the template; 0 if either image is degenerate;
 *   fwhm [2, 3] float32 (nullable): full width at half maximum in degrees of
 *     each curve (row 0 NDP, row 1 FFT; columns x, y, z): half = max / 2, the
 *     crossings nearest the maximum (the lowest-index maximum) placed by linear
 *     interpolation, -1 where the curve does not fall below half on both sides
 *     within the scan.
 * 1 <= h <= 2048, step_deg > 0; the master and its size as xcf_project. */
int xcf_rotation_scan(xcf_ctx *ctx, const float *master, int32_t M, const xcf_geometry *g, const double *q,
                      const double *pc_test, int32_t h, double step_deg, float *ndp, float *xcf, float *fwhm,
                      void *stream);

/* SO(3) library generator (paper, "SO(3) Library Generation": the S^2 x S^1
 * scheme of MTEX): the polar angle split into round(pi / d) equal steps, ring
 * i sampled at max(1, round(2 pi sin(Phi_i) / d)) azimuths (half a step
 * offset on odd rings), the rotation about each point split into round(2 pi /
 * d) steps, d = step_deg; orientation = Bunge (azimuth, Phi, rotation) as a
 * unit quaternion (w >= 0); kept where it lies in the cubic (432) fundamental
 * zone (faces included), in generation order (ring, azimuth, rotation).
 * With XCF_SO3_DEDUP a point within 1e-3 deg of an earlier in-zone point (a
 * symmetry copy across a face) is dropped.  Rounding: halves away from zero.
 *   *count (host) receives the number of orientations; quats [cap, 4] float64
 *   (device, NULL to query the count) receives them; XCF_ERR_SIZE if cap is
 *   smaller than the count.  0.5 <= step_deg <= 180.  Synchronous. */
#define XCF_SO3_DEDUP 1
int xcf_so3_grid(xcf_ctx *ctx, double step_deg, int32_t flags, double *quats, int64_t cap, int64_t *count,
                 void *stream);

/* Nearest neighbour under the cubic disorientation (the second Eq. 6; the
 * Fig. 2 study of a library's spacing): for each qa[i] the qb[j] of smallest
 * disorientation, over every j (mode 0), j != i (mode 1; the sets are one,
 * qb may be NULL = qa) or j < i (mode 2).  Pairs are ranked in FP32 (ties ->
 * lowest j); the chosen pair's angle is recomputed in FP64.
 *   qa [na, 4], qb [nb, 4] float64 unit quaternions (device); angle_deg [na]
 *   float64 and index [na] int32 out (-1 and -1 when there is no candidate). */
int xcf_nearest_disorientation(xcf_ctx *ctx, const double *qa, int32_t na, const double *qb, int32_t nb,
                               int32_t mode, double *angle_deg, int32_t *index, void *stream);

/* Several maps in one search (paper, Fig. 1 B-C, for every map of a batch;
 * the maps may have different detectors, pattern centres and libraries --
 * each map's detector is cropped to its square by the library's crop rule,
 * e.g. 96 -> 64, 160 / 200 -> 128 px, or 96 and 160 kept whole with the
 * native rule).  Patterns are pre-processed per map, then every map up to
 * 160 x 160 is searched in ONE persistent launch (one 512-thread CTA per SM)
 * that takes (map, pattern, template range) work items of all sides from one
 * queue; 256 x 256 maps (four-CTA clusters) and native 200 x 200 maps (one
 * template per pass through the real-output transform) run their own search
 * kernels in the same stream.  For each (detector side, library size) the
 * search body and the work granularity are chosen by timing candidates on the
 * first call (cached in the context; see xcf_maps_get_tuning): the body is one
 * of the line-transform decompositions the queue has for that side,
 *   XCF_BODY_REG     rows and columns as warp-line transforms in registers,
 *                    N = R x 32 points (64, 96, 128, 160): R points per lane,
 *                    five 32-point lane stages by shuffles;
 *   XCF_BODY_ROUNDS  N = 128 only: three register rounds (16-point column
 *                    FFTs; radix 8 + radix 4; 32-point row FFTs) with two
 *                    shared-memory transposes (the kernel of xcf_index);
 *   XCF_BODY_SMEM    N = 16, 32, 64: the surface in shared memory, radix-2
 *                    line transforms;
 *   XCF_BODY_OCT     N = 64 only: eight-lane groups, a 64-point line as an
 *                    8-point FFT in registers, a twiddle, a shared-memory
 *                    transpose and a second 8-point FFT (the kernel of
 *                    xcf_index at N = 64);
 * the number of patterns a CTA searches side by side (1, 2 or 4 groups of
 * warps, each with its share of the shared memory, where the body fits), and
 * the granularity, the number of template pairs per work item (the whole
 * library, a quarter or a sixteenth).  With XCF_MAPS_GRAPH the whole
 * sequence is captured in a CUDA graph the first time a batch configuration
 * (pointers and sizes) is seen and replayed afterwards: the patterns may
 * change between calls, the pointers may not.  Outputs per map as xcf_index
 * (the same best template up to ties between bodies: different transform
 * orders round differently).  Asynchronous with respect to `stream` except
 * for the first call of a configuration. */
typedef struct {
    const xcf_library *lib;   /* the map's library (its detector geometry)        */
    const float *patterns;    /* [P, H, W] float32 on the library's detector      */
    int32_t P;
    int32_t *best;            /* [P]                                              */
    float *peak;              /* [P]                                              */
    float *shift;             /* [P, 2]                                           */
} xcf_map_desc;
#define XCF_MAPS_GRAPH 1
int xcf_index_maps(xcf_ctx *ctx, const xcf_map_desc *maps, int32_t n_maps, int32_t flags, void *stream);

#define XCF_BODY_REG 0
#define XCF_BODY_ROUNDS 1
#define XCF_BODY_SMEM 2
#define XCF_BODY_OCT 3
/* The multi-map tuning of (side N, library size T) on ctx: the search body
 * (XCF_BODY_*), the groups per CTA (1, 2 or 4 patterns side by side, each on
 * 512 / groups threads and that share of the shared memory) and the template
 * pairs per work item.  Host only.  get: XCF_ERR_ARG if that (N, T) has not
 * been tuned yet.  set: fixes the choice (pairs clamped to the library's pair
 * count) for later xcf_index_maps calls, instead of timing candidates, and
 * drops the context's captured graph; XCF_ERR_ARG if the body does not serve
 * side N, the groups are not 1, 2 or 4 or do not fit the body's shared
 * memory (XCF_BODY_ROUNDS: 1; XCF_BODY_REG at 128 and 160: 1; at 96: 1 or 2;
 * XCF_BODY_OCT: 1, 2 or 4),
 * or T, pairs <= 0. */
int xcf_maps_get_tuning(const xcf_ctx *ctx, int32_t N, int32_t T, int32_t *body, int32_t *groups,
                        int32_t *pairs);
int xcf_maps_set_tuning(xcf_ctx *ctx, int32_t N, int32_t T, int32_t body, int32_t groups, int32_t pairs);

/* Search then refine in one call (device memory): xcf_index with pcs, seeds =
 * the library orientations of the best templates (identity for degenerate
 * patterns), then xcf_refine with pcs and the context's max_iter / tol_deg.
 * Outputs as those two calls. */
int xcf_index_refine(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                     const double *pcs, int32_t *best, float *peak, float *shift, double *quats,
                     float *rpeak, int32_t *iters, void *stream);

/* End to end from host memory: search and refine P patterns held in host
 * memory (pinned for full speed), streaming them through the device in chunks
 * of `chunk` patterns (<= 0: about four chunks of at least 2,048 patterns;
 * at most 16,384): two device slots, the next chunk's patterns copied in on a
 * copy stream while the current chunk is indexed and refined on a compute
 * stream, and each chunk's outputs copied back behind it.  pcs (host, [P, 3])
 * may be NULL.  Outputs: best, peak, shift as xcf_index with pcs; quats,
 * rpeak, iters as xcf_refine (seeds = library orientations of best, the
 * context's max_iter / tol_deg).  Synchronous. */
int xcf_index_refine_host(xcf_ctx *ctx, const xcf_library *lib, const float *patterns,
                          int32_t P, const double *pcs, int32_t chunk, int32_t *best, float *peak,
                          float *shift, double *quats, float *rpeak, int32_t *iters);

/* Library search without device allocation.  No counterpart in the paper.
 *
 * Some callers cannot call cudaMalloc: code whose device memory is entirely
 * owned by another allocator (e.g. a framework's caching allocator that has
 * reserved the GPU), or a latency-critical loop that cannot accept the
 * device-wide synchronisation of cudaMalloc / cudaFree.  xcf_index_noalloc
 * gives them the results of xcf_index (same kernels, same arguments and
 * outputs) while allocating nothing: its scratch (pattern spectra, flags and
 * keys) lives in one fixed array of XCF_NOALLOC_SCRATCH_BYTES compiled into
 * the library, which every GPU that loads the library holds until the
 * process exits.  The caller still provides inputs and outputs.
 *  - P may not exceed xcf_noalloc_max_patterns(N) (992 patterns at N = 64,
 *    252 at N = 128, 63 at N = 256); larger P fails with XCF_ERR_SIZE and a
 *    message naming the limit.  Every side the library builds is served
 *    (native 96 and 160 included); the up-sampled peak option is not
 *    (XCF_ERR_UNIMPLEMENTED: it needs scratch).
 *  - The array is committed on a device by the first call there, not when
 *    the library is loaded: CUDA loads the library's modules lazily by
 *    default, and that first call loads the module holding the array (and
 *    looks up its device address, once per device and CUDA context).  So
 *    the first call on each device commits XCF_NOALLOC_SCRATCH_BYTES plus
 *    the module's small code, and can fail with XCF_ERR_CUDA when the GPU is
 *    full.  Make it before another allocator reserves the GPU, and before
 *    any stream capture; later calls allocate nothing.
 *  - All calls on a device share the one array and it keeps the previous
 *    call's contents (the call clears what must start at zero).  Calls whose
 *    work overlaps on the GPU (other streams, other host threads) race on it:
 *    serialise them. */
#define XCF_NOALLOC_SCRATCH_BYTES (16u << 20)
int xcf_index_noalloc(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                      int32_t *best, float *peak, float *shift, void *stream);

/* Measured FP32 FMA throughput of the context's device (the paper has no
 * counterpart: a measurement utility).  The all-pairs search is bound by FP32
 * arithmetic, and its roofline takes SMs x 128 FMA lanes x 2 flops x clock as
 * the peak; this launches 4 x SMs CTAs of 1,024 threads, each thread running
 * eight independent FMA chains of 65,536 FMAs, and reports the best of three
 * timed launches: tflops = flops / time in TFLOP/s, ms (nullable) the launch
 * time.  Synchronous with respect to `stream`.                              */
int xcf_fp32_fma_rate(xcf_ctx *ctx, double *tflops, double *ms, void *stream);

/* Largest P that xcf_index_noalloc accepts for detector side n (0 if n is
 * not a side the kernels take: 16, 32, 64, 96, 128, 160, 256).  Host only. */
int xcf_noalloc_max_patterns(int32_t n);

/* ---------------------------------------------------------------------
 * Learned orientation proposal.  An extension of the paper's method: a small
 * convolutional network proposes k orientations per pattern, each proposal is
 * scored by the cross-correlation peak of its reprojected template (Fig. 1
 * B-C), the best is refined (Fig. 6, Eq. 7), and patterns whose refined peak
 * stays below a threshold fall back to the full library search.
 *
 * Network (input: the centred 128 x 128 crop of the detector, standardised
 * per pattern): five 3 x 3 stride-2 convolutions with bias and ReLU, channels
 * 1 -> 32 -> 64 -> 64 -> 128 -> 128; mean pool; fc 128 -> 256 + ReLU; fc
 * 256 -> 6k.  Head h maps its six outputs (a1, a2) to the rotation with
 * columns b1 = a1/|a1|, b2 = normalised a2 - (b1.a2) b1, b3 = b1 x b2.
 * Training loss per pattern: min over heads and the 24 cubic operators S of
 * |R_h - S R(q_gt)|_F^2; the batch loss is the mean.  Parameters: one float
 * array, blocks conv1 W [32][1][3][3], b [32], ..., conv5 W, b, fc1 W [256][128],
 * b [256], fc2 W [6k][256], b [6k].  FP32 throughout.
 * --------------------------------------------------------------------- */
typedef struct xcf_net xcf_net;
#define XCF_NET_SIDE 128

/* Parameter count for k heads (1 <= k <= 64), -1 otherwise.  Host only. */
int64_t xcf_net_num_params(int32_t k);

/* Network with k heads on the context's device.  params: device [n] copied in,
 * or NULL for all zeros.  Adam state starts at zero.  Synchronous. */
int xcf_net_create(xcf_ctx *ctx, int32_t k, const float *params, xcf_net **out);
int xcf_net_free(xcf_net *net);

/* Device pointer to the parameters (owned by the net, writable) and their count. */
int xcf_net_params(xcf_net *net, float **params, int64_t *n);

/* Raw outputs out [B][6k] for images [B][H][W] on detector g (the net reads the
 * centred 128 x 128 crop; XCF_ERR_SIZE if the detector is smaller), or
 * [B][128][128] when g is NULL. */
int xcf_net_forward(xcf_ctx *ctx, xcf_net *net, const float *images, int32_t B, const xcf_geometry *g,
                    float *out, void *stream);

/* Mean loss of the batch (loss: device double [1], written) and its gradient
 * kept in the net for xcf_net_adam (also copied to grad [n] when non-NULL);
 * winners [B][2] (head, cubic operator index; may be NULL).  quats_gt [B][4]. */
int xcf_net_loss_grad(xcf_ctx *ctx, xcf_net *net, const float *images, int32_t B, const xcf_geometry *g,
                      const double *quats_gt, double *loss, float *grad, int32_t *winners, void *stream);

/* One Adam step (Kingma & Ba 2015) with the gradient of the last
 * xcf_net_loss_grad: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
int xcf_net_adam(xcf_ctx *ctx, xcf_net *net, float lr, float beta1, float beta2, float eps, void *stream);

/* Inference precision of the network's forward pass in xcf_net_forward,
 * xcf_propose and xcf_index_learned: on = 0 FP32 (default); on = 1 the
 * convolutions after the first on the tensor cores with BF16 operands (layer
 * inputs and weights rounded to BF16) and FP32 accumulation.  Training
 * (xcf_net_loss_grad) always runs in FP32.  With BF16 on, those calls wait
 * for the device at their end to read the tensor-core status word
 * (XCF_ERR_TIMEOUT if a bounded wait gave up).  Host only. */
int xcf_net_set_bf16(xcf_net *net, int32_t on);

/* k proposals per pattern: quats [P][k][4] (unit, w >= 0). */
int xcf_propose(xcf_ctx *ctx, xcf_net *net, const float *patterns, int32_t P, const xcf_geometry *g,
                double *quats, void *stream);

/* Learned indexing: proposals, correlation score of each (the best by peak;
 * ties to the lowest head), refinement of the best, then for every
 * non-degenerate pattern whose refined peak is below tau the full search over
 * lib and refinement from its best template.  Outputs as xcf_refine, plus
 * fallback [P] (1 where the full search ran).  The library needs its master
 * pattern.  Synchronises once per chunk of patterns (to size the fallback). */
int xcf_index_learned(xcf_ctx *ctx, xcf_net *net, const xcf_library *lib, const float *patterns, int32_t P,
                      const double *pcs, float tau, double *quats, float *peak, int32_t *iters, int32_t *fallback,
                      void *stream);

/* Profiling.  Every context counts the kernels it launches, per stage.  When
 * timing is enabled it also records a CUDA event pair on the launching stream
 * around each launch and accumulates the elapsed device time per stage. */
#define XCF_STAGE_PROJECT  0   /* gnomonic reprojection                          */
#define XCF_STAGE_PREP     1   /* crop, standardise, window, FFT, filter, norm    */
#define XCF_STAGE_SEARCH   2   /* all-pairs correlation and best-template keys    */
#define XCF_STAGE_PEAK     3   /* single-surface argmax and sub-pixel fit         */
#define XCF_STAGE_LOGPOLAR 4   /* log-polar resampling                            */
#define XCF_STAGE_UPDATE   5   /* refinement updates (X/Y shift, angular xcf + Z) */
#define XCF_STAGE_OTHER    6   /* small bookkeeping kernels                       */
#define XCF_STAGE_SCREEN   7   /* tensor-core zero-shift screen (GEMM)            */
#define XCF_STAGE_NET      8   /* proposal network: forward, backward, optimiser  */
#define XCF_NUM_STAGES     9

/* Cap the context's device scratch (the sum of its grow-only buffers) at
 * `bytes` (0 = no cap).  A call that would grow the scratch past the cap
 * fails with XCF_ERR_OOM before allocating, and the context stays usable (for
 * calls that fit, or after raising the cap).  Lets a caller share the device
 * with other work, and lets tests exercise the out-of-memory path without
 * exhausting the device.  Host only. */
int xcf_set_scratch_limit(xcf_ctx *ctx, uint64_t bytes);

/* Bytes of device scratch the context holds now.  Host only. */
int xcf_scratch_bytes(const xcf_ctx *ctx, uint64_t *bytes);

/* Turn event timing on (1) or off (0).  Host only. */
int xcf_profile_enable(xcf_ctx *ctx, int on);

/* Per-stage accumulated device milliseconds (ms, may be NULL) and kernel
 * launch counts (launches, may be NULL), arrays of XCF_NUM_STAGES.  Waits for
 * the recorded events.  reset != 0 clears the accumulators afterwards. */
int xcf_profile_read(xcf_ctx *ctx, double *ms, int64_t *launches, int reset);

#ifdef __cplusplus
}
#endif
#endif /* EBSDXCF_H */
