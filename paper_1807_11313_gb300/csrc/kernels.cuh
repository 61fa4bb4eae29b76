// Launchers of the ebsdxcf kernels (host side, internal to the library).
// Every launcher enqueues on `st` and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct PrepArgs {
    int N;            // square side after the crop
    int W, H;         // detector (source image) size
    int ox, oy;       // crop offsets
    int window;       // 0 none, 1 Hann
    float inv2shp;    // 1 / (2 sigma_hp^2)
    float inv2slp;    // 1 / (2 sigma_lp^2)
};

struct ProjArgs {
    int W, H;                 // detector size
    int ox, oy, nx, ny;       // output region: detector pixels [oy, oy+ny) x [ox, ox+nx)
    double pcx, pcy, pcz;     // default pattern centre (when pcs == nullptr)
    double alpha;             // detector -> sample rotation about x, radians
    int interp = 0;           // master lookup: 0 bilinear, 1 bicubic (Keys)
    double ca = 1.0, sa = 0.0;   // cos / sin of alpha (set by launch_project)
};

// pre-processing: images [P, H, W] -> half spectra [P, N, N/2+1] (+ spatial [P, N, N])
// `active` (nullable): images whose flag is 0 are skipped entirely
cudaError_t launch_prep(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial,
                        int *degen, const int *active, cudaStream_t st);
// images made by projecting the master pattern instead of read from memory:
// image p is the projection of region `a` (nx x ny = the image's W x H) at
// orientation quats[p] and pattern centre pcs[p] (or a's default)
struct ProjSrc {
    const float *master = nullptr;
    int M = 0;
    const double *quats = nullptr;   // [P][4]
    const double *pcs = nullptr;     // [P][3] or null
    ProjArgs a;
};
// pre-processing of projected images (launch_project then launch_prep, in one
// kernel and without the images in memory): sides 16, 32, 64 and 128;
// cudaErrorNotSupported for the others
cudaError_t launch_prep_projected(const ProjSrc &src, int P, const PrepArgs &a, float2 *spec, float *spatial,
                                  int *degen, const int *active, cudaStream_t st);

// all-pairs search: per-pattern best key (atomicMax) and optional per-pair peaks [P, T]
cudaError_t launch_search(int N, const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                          unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st);

// N = 256 search on clusters of four CTAs (the 256 x 256 array in distributed
// shared memory); St: the templates in the search layout (launch_pack_c256),
// Sp: the patterns' half spectra; with cand: each pattern's candidate list
// cand [P][kc]
cudaError_t launch_search_c256(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                               unsigned long long *keys, float *peaks_all, const int *cand, int kc,
                               cudaStream_t st);
// the N = 256 search layout: float2 per template, and the packing of T half spectra
size_t c256_search_layout_f2();
cudaError_t launch_pack_c256(const float2 *spectra, int T, float2 *packed, cudaStream_t st);
// N = 256 single-surface peak on clusters of four CTAs (two patterns per pass)
cudaError_t launch_pair_peak_c256(const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                  const int *active, int P, float *peak, float *shift, cudaStream_t st,
                                  int *argmax = nullptr);
// N = 256 pre-processing on clusters of four CTAs (one image per cluster)
cudaError_t launch_prep_c256(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                             const int *active, cudaStream_t st);

// search over each pattern's candidate list cand [P][kc] (library indices, < 0 empty)
cudaError_t launch_search_list(int N, const float2 *St, const int *cand, int kc, const float2 *Sp,
                               const int *degen, int P, unsigned long long *keys, float *peaks, int num_sms,
                               cudaStream_t st);

// BF16 zero-shift screen S[P][T] = A[P][K] . B[T][K]^T on tcgen05; err set on a timed-out wait
cudaError_t launch_screen_tc(const void *A, int P, const void *B, int T, int K, float *S, int *err,
                             cudaStream_t st);
// top-k (k <= 64) of each row of S [P][T]: candidates by (score desc, index asc)
cudaError_t launch_topk_rows(const float *S, int P, int T, int k, int *cand, float *score, cudaStream_t st);
cudaError_t launch_to_bf16(const float *x, size_t n, void *y, cudaStream_t st);

// multi-map search: one persistent launch over a queue of work items
// search bodies of the multi-map queue (values of XCF_BODY_* in the header)
constexpr int kBodyReg = 0;      // register warp-line transforms (N = R x 32: 64, 96, 128, 160)
constexpr int kBodyRounds = 1;   // N = 128: three register rounds with two shared-memory transposes
constexpr int kBodySmem = 2;     // surface in shared memory, radix-2 line transforms (2^k sides up to 64)
constexpr int kBodyOct = 3;      // N = 64: eight-lane groups, 8 x 8 line transforms with shared-memory transposes
constexpr int kNumBodies = 4;
struct MapDev {
    int N, T, body;                // detector side, library size, search body (items of the map run on
                                   // groups of 512 / G threads, G from the map's phase of the queue)
    const float2 *St;              // library half spectra [T][N][N/2+1]
    const float2 *Stp;             // N = 128: the same in the packed layout of the three-round body
    const float2 *Sp;              // the map's pattern spectra
    const int *degen;              // the map's degeneracy flags
    unsigned long long *keys;      // the map's best keys
};
// whether the queue serves side N with body b
__host__ __device__ inline bool body_serves(int N, int b) {
    if (b == kBodyReg) return N == 64 || N == 96 || N == 128 || N == 160;
    if (b == kBodyRounds) return N == 128;
    if (b == kBodySmem) return N == 16 || N == 32 || N == 64;
    if (b == kBodyOct) return N == 64;
    return false;
}
struct WorkItem {
    int map, p, pb, pe;            // pattern p of map `map` against template pairs [pb, pe)
};
size_t maps_smem_bytes();
constexpr int kMapsThreads = 512;   // threads of a queue CTA
// shared memory one item of side N with body b needs on nt threads (the queue
// gives each of the G groups of a CTA maps_smem_bytes() / G, rounded down to
// 16 bytes, and 512 / G threads)
inline size_t maps_item_smem(int N, int b, int nt = kMapsThreads) {
    if (b == kBodyRounds) return (size_t)8 * (128 * 65 + 128 * 128 + 128 + 128 + 256 + 32 + 128);
    if (b == kBodyOct) return (size_t)8 * (64 * 64 + (size_t)(nt / 8) * 72 + 16);
    return (size_t)8 * ((size_t)N * (N + 1) + N + 34);
}
// Items are ordered by phase: [offs[0], offs[1]) run on whole CTAs, [offs[1],
// offs[2]) on two groups of 256 threads per CTA, [offs[2], offs[3]) on four
// groups of 128.  grid > 0: persistent CTAs, each phase's items taken from its
// own atomic counter (counters[0..2]); grid <= 0: one CTA per 1, 2 or 4 items.
cudaError_t launch_search_maps(const MapDev *maps, const WorkItem *items, const int offs[4], int *counters,
                               int grid, cudaStream_t st);

// N = 128: library half spectra -> the search kernel's packed layout
cudaError_t launch_pack_search_layout(const float2 *spectra, int T, int N, float2 *packed, cudaStream_t st);

// peak of one surface per pattern: template spectrum = St + (tidx ? tidx[p] : p) * H;
// argmax (nullable) receives the integer peak's row-major index
cudaError_t launch_pair_peak(int N, const float2 *St, const int *tidx, const float2 *Sp,
                             const int *degen, const int *active, int P, float *peak, float *shift,
                             cudaStream_t st, int *argmax = nullptr);
// up-sampled peak (U >= 2): the correlation's Fourier series on a +-1 px grid of step 1/U
// around argmax[p]; overwrites peak and shift of every computed pattern
cudaError_t launch_upsample_peak(int N, const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                 const int *active, int P, int U, const int *argmax, float *peak, float *shift,
                                 cudaStream_t st);

cudaError_t launch_keys_to_best(const unsigned long long *keys, int P, int *best, cudaStream_t st);

cudaError_t launch_project(const float *master, int M, const double *quats, const double *pcs,
                           const int *active, int P, const ProjArgs &a, float *out, cudaStream_t st);

cudaError_t launch_logpolar(const float *spatial, const int *active, int P, int N, int nr, int neta,
                            float rmin, float rmax, float *out, cudaStream_t st);

// refinement updates (float64 orientation algebra)
cudaError_t launch_update_xy(const double *q, const float *shift, const double *pcs, double pcz_def,
                             int W, double alpha, const int *active, int P, double *q1,
                             cudaStream_t st);
// windows: radial bands of the log-polar images (1 .. min(16, nr)), each
// correlated along eta on its own; the update takes the median band shift
cudaError_t launch_eta_update(const float *lpT, const float *lpP, int nr, int neta, int windows,
                              const double *q0, const double *q1, double alpha, double tol_deg, int *active,
                              int *iters, double *q_out, int P, cudaStream_t st);

cudaError_t launch_gather_seeds(const double *lib_quats, const int *best, int P, double *seeds,
                                cudaStream_t st);
// select (nullable): patterns with select[p] == 0 are not refined and their outputs are left untouched
cudaError_t launch_shift_pc(const double *pcs, double pcx, double pcy, int W, int H, const int *best, int P,
                            float *shift, cudaStream_t st);
cudaError_t launch_init_refine(const int *degen, const int *select, int P, int *active, int *iters, float *peak,
                               cudaStream_t st);
cudaError_t launch_copy_active_peak(const float *src, const int *active, int P, float *dst,
                                    cudaStream_t st);
cudaError_t launch_disorientation(const double *qa, const double *qb, int n, double *out,
                                  cudaStream_t st);

// normalised dot product (Eq. 1): contrast-normalised crops / sqrt(d) of
// images [P] (image p at img + p * img_stride, rows row_stride apart, crop at
// (ox, oy), side n a power of two) -> out32 [P][n*n] and / or out16 (BF16), degen [P]
cudaError_t launch_ndp_norm(const float *img, int P, long img_stride, int row_stride, int ox, int oy, int n,
                            float *out32, void *out16, int *degen, cudaStream_t st);
// background correction of the same crops: out [P][n][n] = crop - Gaussian
// blur (sigma px, 0 < sigma <= n), tmp [P][n][n] work array
cudaError_t launch_ndp_background(const float *img, int P, long img_stride, int row_stride, int ox, int oy, int n,
                                  float sigma, float *tmp, float *out, cudaStream_t st);
// FP32 NDP of pattern p (pn [P][d]) against its candidates cand [P][k] of
// tn [T][d] (< 0 skipped): best [P] (-1 if degenerate), score [P]
cudaError_t launch_ndp_rescore(const float *pn, const float *tn, long d, const int *cand, int k, const int *degen,
                               int P, int *best, float *score, cudaStream_t st);
// FWHM of nc curves of length L (the first nc/2 from a, the rest from b) -> out [nc]
cudaError_t launch_fwhm(const float *a, const float *b, int nc, int L, float step, float *out, cudaStream_t st);
// rotation experiment: qs [1 + 3L][4], pcs [1 + 3L][3] (detector-frame PCs), L = 2h + 1
cudaError_t launch_scan_setup(const double *q, const double *pc_test, double pcx, double pcy, double pcz, int h,
                              double step_rad, double alpha, double *qs, double *pcs, cudaStream_t st);

// SO(3) library generator: grid point g of ring i (ring_start [n_rings], ring_az
// [n_rings] azimuths) -> q_all [G][4] and its cubic-zone flag [G]
cudaError_t launch_so3_points(const long long *ring_start, int n_rings, int n_polar, int n_s1, const int *ring_az,
                              long long G, double *q_all, int *flag, cudaStream_t st);
// order-preserving compaction of the flagged rows of q_in [G][4] -> q_out (nullable:
// count only); block_counts [compact_blocks(G)], *total (device) = the count
int compact_blocks(long long G);
cudaError_t launch_compact(const double *q_in, const int *flag, long long G, int *block_counts, long long *total,
                           double *q_out, cudaStream_t st);
// flag[i] = 0 where 0 <= angle[i] < thr, else 1
cudaError_t launch_keep_flags(const double *angle, long long n, double thr, int *flag, cudaStream_t st);
// nearest qb of each qa under the cubic disorientation (mode 0 all, 1 j != i,
// 2 j < i): angle [na] degrees (-1 none), index [na]; keys [na] work array
cudaError_t launch_nearest_disorientation(const double *qa, int na, const double *qb, int nb, int mode,
                                          unsigned long long *keys, double *angle, int *index, int num_sms,
                                          cudaStream_t st);

// ------------------------------------------------ learned proposal network
// input images: the 128 x 128 crop at (ox, oy) of image b = x + b * img_stride
struct CnnInput {
    const float *x;
    long img_stride, row_stride;
    int ox, oy;
};
long cnn_num_params(int k);
size_t cnn_act_floats(int B, int k);    // activations of a batch (forward, kept for backward)
size_t cnn_grad_floats(int B, int k);   // gradient work buffers of a batch
const float *cnn_output(float *act, int B, int k);   // [B][6k] inside the activations
// BF16 inference form: convolutions 2..5 on the tensor cores (BF16 operands,
// FP32 accumulation); the same outputs location; work: cnn_bf16_work_bytes(B)
// bytes (256-byte aligned); err: the tensor-core pipeline's status word
size_t cnn_bf16_work_bytes(int B);
cudaError_t launch_cnn_forward_bf16(const float *params, int k, const CnnInput &in, int B, float *act, void *work,
                                    int *err, int num_sms, int *launches, cudaStream_t st);
// convolution `layer` (1..4 = the network's second to fifth) as an implicit
// GEMM on the tensor cores: x NHWC BF16 [B][S][S][Ci], w BF16 [Co][Kp] in the
// order (ky * 3 + kx) Ci + ci (zero beyond 9 Ci), y NHWC [B][S/2][S/2][Co] =
// relu(conv + bias), BF16 for layers 1..3 and FP32 for layer 4; (Ci, Co, S) =
// (32, 64, 64), (64, 64, 32), (64, 128, 16), (128, 128, 8); err set to 1 when
// a pipeline wait expired; x, w, y 16-byte aligned
cudaError_t launch_conv_tc(int layer, const void *x, int B, const void *w, const float *bias, void *y, int *err,
                           int num_sms, cudaStream_t st);
cudaError_t launch_cnn_forward(const float *params, int k, const CnnInput &in, int B, float *act, int *launches,
                               cudaStream_t st);
// after launch_cnn_forward on the same act: loss_sum += sum of per-pattern
// losses, grad = d(mean loss)/d(params), winners [B][2] (nullable)
cudaError_t launch_cnn_backward(const float *params, int k, const CnnInput &in, int B, float *act, float *gbuf,
                                const double *qgt, double *loss_sum, int *winners, float *grad, int num_sms,
                                int *launches, cudaStream_t st);
cudaError_t launch_cnn_proposals(const float *out, int n_heads_total, double *quats, cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, long n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t st);
cudaError_t launch_take_head(const double *prop, int P, int k, int h, double *q, cudaStream_t st);
cudaError_t launch_keep_best(const float *peak_h, const double *q_h, int P, int h, float *best_peak, double *best_q,
                             int *best_h, cudaStream_t st);
cudaError_t launch_fallback_flags(const float *peak, const int *degen, int P, float tau, int *fb, int *count,
                                  cudaStream_t st);
cudaError_t launch_fallback_mask(const int *degen, const int *fb, int P, int *mask, cudaStream_t st);
// the fallback pass on the flagged patterns, gathered by pattern pairs (each
// keeps its pair-peak partner): the ordered pair list (P <= 2 x 1024 x 1024;
// idx and flag_c of 2 x pairs entries, pairs[0] = count), row gathers, seeds
// (library orientation of the best template for flagged patterns, else the
// current one) and the flagged patterns' results scattered back
cudaError_t launch_fallback_list(const int *fb, int P, int *idx, int *flag_c, int *pairs, cudaStream_t st);
cudaError_t launch_gather_rows(const float *src, size_t len, const int *idx, int n, float *dst, cudaStream_t st);
cudaError_t launch_gather_rows(const double *src, size_t len, const int *idx, int n, double *dst, cudaStream_t st);
cudaError_t launch_fallback_seeds_list(const int *idx, const int *flag_c, const int *best, const double *lib_q,
                                       const double *cur, int n, double *seeds, cudaStream_t st);
cudaError_t launch_fallback_scatter(const int *idx, const int *flag_c, int n, const double *q_c, const float *peak_c,
                                    const int *it_c, double *q, float *peak, int *iters, cudaStream_t st);
cudaError_t launch_fallback_seeds(const int *fb, const int *best, const double *lib_q, const double *cur, int P,
                                  double *seeds, cudaStream_t st);

// FP32 FMA rate probe (k_peak.cu): flops of one launch of the given shape
cudaError_t launch_fma_rate(int blocks, int threads, int iters, float *sink, cudaStream_t st);
double fma_rate_flops(int blocks, int threads, int iters);

// the native 200 x 200 side (k_n200.cu): pre-processing, the all-pairs search
// (cand != null: each pattern's candidate list of kc library indices) and the
// single-surface peak, with the arguments of the launchers above
cudaError_t launch_prep_n200(const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial, int *degen,
                             const int *active, cudaStream_t st);
cudaError_t launch_search_n200(const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                               unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st,
                               const int *cand, int kc);
cudaError_t launch_pair_peak_n200(const float2 *St, const int *tidx, const float2 *Sp, const int *degen,
                                  const int *active, int P, float *peak, float *shift, int *argmax, cudaStream_t st);
