// Host side of the ebsdxcf C ABI: argument checks, the per-context scratch
// arena, library construction, and the index / refine / end-to-end flows.
// Every compute step is one of the kernels in this directory; the host only
// sequences launches on the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/ebsdxcf.h"
#include "internal.h"
#include "kernels.cuh"

using namespace xcf_internal;

namespace {

int fail(xcf_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(xcf_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? XCF_ERR_OOM : XCF_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define XCF_CHECK(expr, where)                                  \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

// a kernel launch of `stage` on stream `st`: counted, and timed with an
// event pair when the context's timing is on
#define XCF_LAUNCH(stage, st, expr, where)                                   \
    do {                                                                     \
        cudaEvent_t a_ = nullptr, b_ = nullptr;                              \
        if (ctx->timing && cudaEventCreate(&a_) == cudaSuccess)              \
            cudaEventRecord(a_, st);                                         \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) {                                             \
            if (a_) cudaEventDestroy(a_);                                    \
            return cuda_fail(ctx, e_, where);                                \
        }                                                                    \
        ctx->launches[stage] += 1;                                           \
        if (a_ && cudaEventCreate(&b_) == cudaSuccess) {                     \
            cudaEventRecord(b_, st);                                         \
            ctx->recs.push_back({stage, a_, b_});                            \
        } else if (a_) {                                                     \
            cudaEventDestroy(a_);                                            \
        }                                                                    \
    } while (0)

// a captured multi-map graph holds scratch pointers: it dies with them
void drop_graph(xcf_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    ctx->graph_key.clear();
}

// grow-only scratch buffer; cudaFree / cudaMalloc synchronise, so the first
// call at a size pays for it and later calls reuse the allocation
int scratch(xcf_ctx *ctx, int slot, size_t bytes, void **out) {
    if (bytes == 0) bytes = 16;
    if (ctx->cap[slot] < bytes) {
        if (ctx->scratch_limit) {   // the caller's cap on the arena (0 = none)
            size_t total = bytes;
            for (int i = 0; i < S_COUNT; ++i)
                if (i != slot) total += ctx->cap[i];
            if (total > ctx->scratch_limit)
                return fail(ctx, XCF_ERR_OOM, "scratch of " + std::to_string(bytes) +
                                                  " bytes would exceed the context's limit");
        }
        drop_graph(ctx);
        if (ctx->buf[slot]) cudaFree(ctx->buf[slot]);
        ctx->buf[slot] = nullptr;
        ctx->cap[slot] = 0;
        cudaError_t e = cudaMalloc(&ctx->buf[slot], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, XCF_ERR_OOM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
        }
        ctx->cap[slot] = bytes;
    }
    *out = ctx->buf[slot];
    return XCF_OK;
}

template <typename T>
int scratch_t(xcf_ctx *ctx, int slot, size_t count, T **out) {
    void *p = nullptr;
    int rc = scratch(ctx, slot, count * sizeof(T), &p);
    *out = static_cast<T *>(p);
    return rc;
}

struct Crop {
    int n, ox, oy;
    double pc[3];
};

// centred square crop: the largest 2^k side (native: the largest of 16, 32,
// 64, 96, 128, 160, 256) that fits the detector and cap, PC updated
int crop_of(const xcf_geometry *g, int cap, Crop *c, bool native = false) {
    if (!g || g->width <= 0 || g->height <= 0) return XCF_ERR_ARG;
    int m = g->width < g->height ? g->width : g->height;
    int n = 1;
    if (native) {
        static const int sides[8] = {16, 32, 64, 96, 128, 160, 200, 256};
        n = 0;
        for (int i = 0; i < 8; ++i)
            if (sides[i] <= m && sides[i] <= cap) n = sides[i];
    } else {
        while (n * 2 <= m && n * 2 <= cap) n *= 2;
    }
    if (n < 16) return XCF_ERR_SIZE;
    c->n = n;
    c->ox = (g->width - n) / 2;
    c->oy = (g->height - n) / 2;
    c->pc[0] = (g->pcx * g->width - c->ox) / n;
    c->pc[1] = (g->pcy * g->height - c->oy) / n;
    c->pc[2] = g->pcz * g->width / n;
    return XCF_OK;
}

double alpha_of(const xcf_geometry *g) {
    return (90.0 - g->sample_tilt_deg + g->detector_tilt_deg) * kPi / 180.0;
}

struct Resolved {
    int window;
    double sigma_hp, sigma_lp;
    int nr, neta;
    double rmin, rmax;
    int windows;   // radial log-polar windows of the Z step
};

Resolved resolve(const xcf_options &o, int n) {
    Resolved r;
    r.window = o.window;
    r.sigma_hp = o.sigma_hp > 0 ? o.sigma_hp : 2.0;
    r.sigma_lp = o.sigma_lp > 0 ? o.sigma_lp : n / 4.0;
    r.nr = o.lp_nr > 0 ? o.lp_nr : (n / 4 > 2 ? n / 4 : 2);
    r.neta = o.lp_neta;
    if (r.neta <= 0)   // 2N, rounded up to a power of two for the native 96 / 160 sides
        for (r.neta = 1; r.neta < 2 * n; r.neta *= 2) {
        }
    r.rmin = o.lp_rmin > 0 ? o.lp_rmin : n / 4.0;
    r.rmax = o.lp_rmax > 0 ? o.lp_rmax : n / 2.0 - 1.0;
    r.windows = o.lp_windows > 0 ? o.lp_windows : 4;
    if (r.windows > r.nr) r.windows = r.nr;
    return r;
}

// background sigma of the NDP for side n (0 = no correction)
float ndp_sigma(const xcf_options &o, int n) {
    if (o.ndp_bg_sigma < 0) return 0.f;
    const double s = o.ndp_bg_sigma > 0 ? o.ndp_bg_sigma : n / 8.0;
    return (float)(s < n ? s : n);
}

// contrast-normalised (and, with the background option, first background-
// corrected) crops of P images -> out32 / out16 (NDP operands)
int ndp_operands(xcf_ctx *ctx, const float *img, int P, long img_stride, int row_stride, int ox, int oy, int n,
                 float *out32, void *out16, int *degen, cudaStream_t st) {
    if (n & (n - 1)) return fail(ctx, XCF_ERR_UNIMPLEMENTED, "the NDP needs a 2^k detector side");
    const float sg = ndp_sigma(ctx->opt, n);
    if (sg > 0.f) {
        float *tmp, *cor;
        int rc;
        if ((rc = scratch_t(ctx, S_BG_TMP, (size_t)n * n * P, &tmp)) ||
            (rc = scratch_t(ctx, S_BG_OUT, (size_t)n * n * P, &cor)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_PREP, st, launch_ndp_background(img, P, img_stride, row_stride, ox, oy, n, sg, tmp, cor, st),
                   "ndp background");
        img = cor;
        img_stride = (long)n * n;
        row_stride = n;
        ox = oy = 0;
    }
    XCF_LAUNCH(XCF_STAGE_PREP, st, launch_ndp_norm(img, P, img_stride, row_stride, ox, oy, n, out32, out16, degen, st),
               "ndp normalise");
    return XCF_OK;
}

PrepArgs prep_args(const xcf_geometry *g, const Crop &c, const Resolved &r) {
    PrepArgs a;
    a.N = c.n;
    a.W = g->width;
    a.H = g->height;
    a.ox = c.ox;
    a.oy = c.oy;
    a.window = r.window;
    a.inv2shp = (float)(1.0 / (2.0 * r.sigma_hp * r.sigma_hp));
    a.inv2slp = (float)(1.0 / (2.0 * r.sigma_lp * r.sigma_lp));
    return a;
}

// square n x n template images on the cropped detector (the source image of
// the pre-processing is then the n x n image itself: W = H = n, no offset)
ProjArgs proj_args_cropped(const xcf_geometry *g, const Crop &c, int interp) {
    ProjArgs a;
    a.interp = interp;
    a.W = g->width;
    a.H = g->height;
    a.ox = c.ox;
    a.oy = c.oy;
    a.nx = c.n;
    a.ny = c.n;
    a.pcx = g->pcx;
    a.pcy = g->pcy;
    a.pcz = g->pcz;
    a.alpha = alpha_of(g);
    return a;
}

PrepArgs prep_args_square(const Crop &c, const Resolved &r) {
    PrepArgs a;
    a.N = c.n;
    a.W = c.n;
    a.H = c.n;
    a.ox = 0;
    a.oy = 0;
    a.window = r.window;
    a.inv2shp = (float)(1.0 / (2.0 * r.sigma_hp * r.sigma_hp));
    a.inv2slp = (float)(1.0 / (2.0 * r.sigma_lp * r.sigma_lp));
    return a;
}

bool supported_n(int n) {
    return n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 200 || n == 256;
}

// pre-processing, search and peak: shared-memory kernels up to N = 160, the
// four-CTA cluster kernels for N = 256
cudaError_t run_prep(xcf_ctx * /*ctx*/, const float *img, int P, const PrepArgs &a, float2 *spec, float *spatial,
                     int *degen, const int *active, cudaStream_t st) {
    if (a.N == 200) return launch_prep_n200(img, P, a, spec, spatial, degen, active, st);
    if (a.N != 256) return launch_prep(img, P, a, spec, spatial, degen, active, st);
    return launch_prep_c256(img, P, a, spec, spatial, degen, active, st);
}

cudaError_t run_search(xcf_ctx * /*ctx*/, int n, const float2 *St, int T, const float2 *Sp, const int *degen, int P,
                       unsigned long long *keys, float *peaks_all, int num_sms, cudaStream_t st) {
    if (n == 200) return launch_search_n200(St, T, Sp, degen, P, keys, peaks_all, num_sms, st, nullptr, 0);
    if (n != 256) return launch_search(n, St, T, Sp, degen, P, keys, peaks_all, num_sms, st);
    return launch_search_c256(St, T, Sp, degen, P, keys, peaks_all, nullptr, 0, st);
}

// templates projected at (quats, pcs) and pre-processed: in one kernel where
// the side has one (the images never reach memory), else the projection into
// img followed by the pre-processing
bool fused_project_prep(int n) { return n == 16 || n == 32 || n == 64 || n == 128; }
int project_prep(xcf_ctx *ctx, const float *master, int M, const double *quats, const double *pcs,
                 const int *active, int P, const ProjArgs &pj, const PrepArgs &ps, float2 *spec, float *spatial,
                 int *degen, float *img, cudaStream_t st) {
    if (fused_project_prep(ps.N)) {
        ProjSrc src;
        src.master = master;
        src.M = M;
        src.quats = quats;
        src.pcs = pcs;
        src.a = pj;
        XCF_LAUNCH(XCF_STAGE_PREP, st, launch_prep_projected(src, P, ps, spec, spatial, degen, active, st),
                   "project + prep templates");
        return XCF_OK;
    }
    XCF_LAUNCH(XCF_STAGE_PROJECT, st, launch_project(master, M, quats, pcs, active, P, pj, img, st), "project");
    XCF_LAUNCH(XCF_STAGE_PREP, st, run_prep(ctx, img, P, ps, spec, spatial, degen, active, st), "prep templates");
    return XCF_OK;
}

// integer peak and 3-point fit, then (with the up-sampling option) the up-sampled peak
cudaError_t run_pair_peak(xcf_ctx *ctx, int n, const float2 *St, const int *tidx, const float2 *Sp,
                          const int *degen, const int *active, int P, float *peak, float *shift, cudaStream_t st) {
    const int U = ctx->opt.upsample;
    int *argmax = nullptr;
    if (U >= 2 && P > 0 && scratch_t(ctx, S_ARGMAX, P, &argmax)) return cudaErrorMemoryAllocation;
    cudaError_t e = n == 200   ? launch_pair_peak_n200(St, tidx, Sp, degen, active, P, peak, shift, argmax, st)
                    : n != 256 ? launch_pair_peak(n, St, tidx, Sp, degen, active, P, peak, shift, st, argmax)
                               : launch_pair_peak_c256(St, tidx, Sp, degen, active, P, peak, shift, st, argmax);
    if (e != cudaSuccess || U < 2) return e;
    return launch_upsample_peak(n, St, tidx, Sp, degen, active, P, U, argmax, peak, shift, st);
}

// spectra: the call correlates against the library's FFT spectra
int check_lib(xcf_ctx *ctx, const xcf_library *lib, bool spectra = false) {
    if (!ctx) return XCF_ERR_ARG;
    if (!lib) return fail(ctx, XCF_ERR_ARG, "library is NULL");
    if (lib->device != ctx->device) return fail(ctx, XCF_ERR_ARG, "library and context on different devices");
    if (spectra && !lib->spectra) return fail(ctx, XCF_ERR_ARG, "library built with XCF_LIB_NO_SPECTRA");
    return XCF_OK;
}

constexpr int kChunk = 16384;   // patterns per pass (bounds the scratch footprint)

// index one chunk already on the device: spectra of the patterns, search,
// best, and the sub-pixel peak of the best template
// only (nullable): patterns with only[p] == 0 are skipped like degenerate ones
// pcs (nullable, [P, 3]): per-pattern pattern centres; the shift is then taken
// relative to the template as it would sit at the pattern's own centre
int index_chunk(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int P, int *best,
                float *peak, float *shift, float *peaks_all, cudaStream_t st, const int *only = nullptr,
                const double *pcs = nullptr) {
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const int H = c.n * (c.n / 2 + 1);
    float2 *sp;
    int *degen;
    unsigned long long *keys;
    int rc;
    if ((rc = scratch_t(ctx, S_SPEC_P, (size_t)P * H, &sp))) return rc;
    if ((rc = scratch_t(ctx, S_DEGEN, P, &degen))) return rc;
    if ((rc = scratch_t(ctx, S_KEYS, P, &keys))) return rc;
    XCF_LAUNCH(XCF_STAGE_PREP, st, run_prep(ctx,patterns, P, prep_args(g, c, r), sp, nullptr, degen, nullptr, st), "prep");
    if (only) {
        int *mask;
        if ((rc = scratch_t(ctx, S_MASK, P, &mask))) return rc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_fallback_mask(degen, only, P, mask, st), "mask");
        degen = mask;
    }
    XCF_CHECK(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * P, st), "memset keys");
    if (peaks_all)   // degenerate patterns keep all-zero rows
        XCF_CHECK(cudaMemsetAsync(peaks_all, 0, sizeof(float) * (size_t)P * lib->T, st), "memset peaks");
    XCF_LAUNCH(XCF_STAGE_SEARCH, st,
               run_search(ctx,c.n, search_spectra(lib), lib->T, sp, degen, P, keys, peaks_all, ctx->num_sms, st),
               "search");
    if (best) {
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_keys_to_best(keys, P, best, st), "keys_to_best");
        XCF_LAUNCH(XCF_STAGE_PEAK, st,
                   run_pair_peak(ctx,c.n, lib->spectra, best, sp, degen, nullptr, P, peak, shift, st),
                   "pair_peak");
        if (pcs)
            XCF_LAUNCH(XCF_STAGE_OTHER, st,
                       launch_shift_pc(pcs, g->pcx, g->pcy, g->width, g->height, best, P, shift, st), "shift_pc");
    }
    return XCF_OK;
}

// max_iter <= 0 / tol_deg < 0: the context's options
int refine_chunk(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int P,
                 const double *seeds, const double *pcs, double *quats, float *peak, int *iters,
                 cudaStream_t st, const int *select = nullptr, bool patterns_ready = false,
                 int max_iter = 0, double tol_deg = -1.0) {
    if (max_iter <= 0) max_iter = ctx->opt.max_iter;
    if (tol_deg < 0.0) tol_deg = ctx->opt.tol_deg;
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const int n = c.n, H = n * (n / 2 + 1), L = r.nr * r.neta;
    float2 *sp, *stt;
    float *yp, *yt, *img, *lpp, *lpt, *shift;
    int *degen, *active;
    double *q1;
    int rc;
    if ((rc = scratch_t(ctx, S_SPEC_P, (size_t)P * H, &sp))) return rc;
    if ((rc = scratch_t(ctx, S_SPEC_T, (size_t)P * H, &stt))) return rc;
    if ((rc = scratch_t(ctx, S_SPATIAL_P, (size_t)P * n * n, &yp))) return rc;
    if ((rc = scratch_t(ctx, S_SPATIAL_T, (size_t)P * n * n, &yt))) return rc;
    if ((rc = scratch_t(ctx, S_IMG, (size_t)P * n * n, &img))) return rc;
    if ((rc = scratch_t(ctx, S_LP_P, (size_t)P * L, &lpp))) return rc;
    if ((rc = scratch_t(ctx, S_LP_T, (size_t)P * L, &lpt))) return rc;
    if ((rc = scratch_t(ctx, S_SHIFT, (size_t)P * 2, &shift))) return rc;
    if ((rc = scratch_t(ctx, S_DEGEN, P, &degen))) return rc;
    if ((rc = scratch_t(ctx, S_ACTIVE, P, &active))) return rc;
    if ((rc = scratch_t(ctx, S_Q1, (size_t)P * 4, &q1))) return rc;
    const PrepArgs pa = prep_args(g, c, r), ps = prep_args_square(c, r);
    const ProjArgs pj = proj_args_cropped(g, c, ctx->opt.master_interp);
    const double alpha = alpha_of(g);
    if (!patterns_ready)   // else sp, yp, degen already hold this chunk's patterns
        XCF_LAUNCH(XCF_STAGE_PREP, st, run_prep(ctx,patterns, P, pa, sp, yp, degen, nullptr, st), "prep patterns");
    XCF_LAUNCH(XCF_STAGE_LOGPOLAR, st,
               launch_logpolar(yp, nullptr, P, n, r.nr, r.neta, (float)r.rmin, (float)r.rmax, lpp, st),
               "logpolar patterns");
    if (quats != seeds)
        XCF_CHECK(cudaMemcpyAsync(quats, seeds, sizeof(double) * 4 * P, cudaMemcpyDeviceToDevice, st),
                  "copy seeds");
    XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_init_refine(degen, select, P, active, iters, peak, st), "init");
    for (int it = 0; it < max_iter; ++it) {
        // X / Y: shift of the template at the current orientation
        if ((rc = project_prep(ctx, lib->master, lib->M, quats, pcs, active, P, pj, ps, stt, nullptr, nullptr, img, st)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_PEAK, st, run_pair_peak(ctx,n, stt, nullptr, sp, degen, active, P, peak, shift, st),
                   "xy peak");
        XCF_LAUNCH(XCF_STAGE_UPDATE, st,
                   launch_update_xy(quats, shift, pcs, g->pcz, g->width, alpha, active, P, q1, st), "xy update");
        // Z: angular shift of the log-polar images
        if ((rc = project_prep(ctx, lib->master, lib->M, q1, pcs, active, P, pj, ps, stt, yt, nullptr, img, st)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_LOGPOLAR, st,
                   launch_logpolar(yt, active, P, n, r.nr, r.neta, (float)r.rmin, (float)r.rmax, lpt, st),
                   "logpolar templates");
        XCF_LAUNCH(XCF_STAGE_UPDATE, st,
                   launch_eta_update(lpt, lpp, r.nr, r.neta, r.windows, quats, q1, alpha, tol_deg, active, iters,
                                     quats, P, st),
                   "z update");
    }
    return XCF_OK;
}

}  // namespace

extern "C" {

const char *xcf_strerror(int code) {
    switch (code) {
        case XCF_OK: return "ok";
        case XCF_ERR_ARG: return "invalid argument";
        case XCF_ERR_SIZE: return "unsupported detector size";
        case XCF_ERR_OOM: return "out of device memory";
        case XCF_ERR_CUDA: return "CUDA error";
        case XCF_ERR_TIMEOUT: return "device wait timed out";
        case XCF_ERR_UNIMPLEMENTED: return "not implemented";
        default: return "unknown error";
    }
}

const char *xcf_last_error(const xcf_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int xcf_options_default(xcf_options *o) {
    if (!o) return XCF_ERR_ARG;
    o->window = 1;
    o->sigma_hp = 2.0;
    o->sigma_lp = 0.0;
    o->lp_nr = 0;
    o->lp_neta = 0;
    o->lp_rmin = 0.0;
    o->lp_rmax = 0.0;
    o->max_iter = 2;
    o->tol_deg = 1e-3;
    o->upsample = 0;
    o->master_interp = 0;
    o->ndp_bg_sigma = 0.0;
    o->lp_windows = 0;
    o->native_sizes = 0;
    return XCF_OK;
}

int xcf_crop(const xcf_geometry *g, int32_t *n, int32_t *off_x, int32_t *off_y, double pc_out[3]) {
    return xcf_crop_ex(g, 0, n, off_x, off_y, pc_out);
}

int xcf_crop_ex(const xcf_geometry *g, int32_t native, int32_t *n, int32_t *off_x, int32_t *off_y,
                double pc_out[3]) {
    if (native != 0 && native != 1) return XCF_ERR_ARG;
    Crop c;
    int rc = crop_of(g, 256, &c, native != 0);
    if (rc) return rc;
    if (n) *n = c.n;
    if (off_x) *off_x = c.ox;
    if (off_y) *off_y = c.oy;
    if (pc_out) memcpy(pc_out, c.pc, sizeof c.pc);
    return XCF_OK;
}

int xcf_create(xcf_ctx **out, const xcf_options *opt, int device) {
    if (!out) return XCF_ERR_ARG;
    *out = nullptr;
    xcf_options o;
    if (opt) {
        o = *opt;
        if (o.window < 0 || o.window > 1 || o.max_iter < 0 || o.sigma_hp < 0) return XCF_ERR_ARG;
        if (o.upsample != 0 && (o.upsample < 2 || o.upsample > 20)) return XCF_ERR_ARG;
        if (o.master_interp < 0 || o.master_interp > 1) return XCF_ERR_ARG;
        if (!(o.ndp_bg_sigma == o.ndp_bg_sigma)) return XCF_ERR_ARG;   // NaN
        if (o.lp_windows < 0 || o.lp_windows > 16) return XCF_ERR_ARG;
        if (o.native_sizes < 0 || o.native_sizes > 1) return XCF_ERR_ARG;
    } else {
        xcf_options_default(&o);
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return XCF_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return XCF_ERR_CUDA;
    }
    xcf_ctx *c = new xcf_ctx();
    c->device = device;
    c->num_sms = sms;
    c->opt = o;
    *out = c;
    return XCF_OK;
}

int xcf_destroy(xcf_ctx *ctx) {
    if (!ctx) return XCF_ERR_ARG;
    cudaSetDevice(ctx->device);
    for (auto &r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    for (auto &e : ctx->gev)
        if (e) cudaEventDestroy(e);
    for (int i = 0; i < S_COUNT; ++i)
        if (ctx->buf[i]) cudaFree(ctx->buf[i]);
    delete ctx;
    return XCF_OK;
}

int xcf_project(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t P,
                const xcf_geometry *g, const double *pcs, float *out, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (P == 0) return XCF_OK;
    if (!master || !quats || !g || !out || P < 0 || M < 2)
        return fail(ctx, XCF_ERR_ARG, "xcf_project: bad argument");
    if (g->width <= 0 || g->height <= 0) return fail(ctx, XCF_ERR_ARG, "xcf_project: bad detector size");
    cudaSetDevice(ctx->device);
    ProjArgs a;
    a.interp = ctx->opt.master_interp;
    a.W = g->width;
    a.H = g->height;
    a.ox = 0;
    a.oy = 0;
    a.nx = g->width;
    a.ny = g->height;
    a.pcx = g->pcx;
    a.pcy = g->pcy;
    a.pcz = g->pcz;
    a.alpha = alpha_of(g);
    cudaStream_t st = (cudaStream_t)stream;
    XCF_LAUNCH(XCF_STAGE_PROJECT, st, launch_project(master, M, quats, pcs, nullptr, P, a, out, st), "project");
    return XCF_OK;
}

int xcf_prep(xcf_ctx *ctx, const float *images, int32_t P, const xcf_geometry *g, float *spectra,
             float *spatial, int32_t *degenerate, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!g || P < 0) return fail(ctx, XCF_ERR_ARG, "xcf_prep: bad argument");
    if (P == 0) return XCF_OK;
    if (!images || !spectra) return fail(ctx, XCF_ERR_ARG, "xcf_prep: bad argument");
    Crop c;
    int rc = crop_of(g, 256, &c, ctx->opt.native_sizes != 0);
    if (rc) return fail(ctx, rc, "xcf_prep: detector too small");
    if (!supported_n(c.n)) return fail(ctx, XCF_ERR_UNIMPLEMENTED, "xcf_prep: detector side not supported");
    cudaSetDevice(ctx->device);
    const Resolved r = resolve(ctx->opt, c.n);
    int *degen = degenerate;
    if (!degen && (rc = scratch_t(ctx, S_DEGEN, P, &degen))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    XCF_LAUNCH(XCF_STAGE_PREP, st,
               run_prep(ctx,images, P, prep_args(g, c, r), reinterpret_cast<float2 *>(spectra), spatial, degen,
                           nullptr, st),
               "prep");
    return XCF_OK;
}

namespace {
int build_from_master(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t T,
                      const xcf_geometry *g, bool spectra, xcf_library **out, void *stream);
int build_from_images(xcf_ctx *ctx, const float *images, const double *quats, int32_t T, const xcf_geometry *g,
                      const float *master, int32_t M, bool spectra, xcf_library **out, void *stream);
}  // namespace

int xcf_build_library(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t T,
                      const xcf_geometry *g, xcf_library **out, void *stream) {
    return build_from_master(ctx, master, M, quats, T, g, true, out, stream);
}

int xcf_build_library_images(xcf_ctx *ctx, const float *images, const double *quats, int32_t T,
                             const xcf_geometry *g, const float *master, int32_t M, xcf_library **out,
                             void *stream) {
    return build_from_images(ctx, images, quats, T, g, master, M, true, out, stream);
}

namespace {
// spectra == false: the library keeps its orientations, master and geometry
// but no FFT spectra (an NDP-only library)
int build_from_master(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t T,
                      const xcf_geometry *g, bool spectra, xcf_library **out, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!master || !quats || !g || !out || T <= 0 || M < 2)
        return fail(ctx, XCF_ERR_ARG, "xcf_build_library: bad argument");
    *out = nullptr;
    Crop c;
    int rc = crop_of(g, 256, &c, ctx->opt.native_sizes != 0);
    if (rc) return fail(ctx, rc, "xcf_build_library: detector too small");
    if (!supported_n(c.n)) return fail(ctx, XCF_ERR_UNIMPLEMENTED, "xcf_build_library: detector side not supported");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Resolved r = resolve(ctx->opt, c.n);
    xcf_library *lib = new xcf_library();
    lib->device = ctx->device;
    lib->T = T;
    lib->N = c.n;
    lib->native = ctx->opt.native_sizes != 0;
    lib->M = M;
    lib->geom = *g;
    lib->ox = c.ox;
    lib->oy = c.oy;
    memcpy(lib->pc, c.pc, sizeof c.pc);
    const size_t H = (size_t)c.n * (c.n / 2 + 1);
    cudaError_t e = spectra ? cudaMalloc(&lib->spectra, sizeof(float2) * H * T) : cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&lib->quats, sizeof(double) * 4 * T);
    if (e == cudaSuccess) e = cudaMalloc(&lib->master, sizeof(float) * 2 * (size_t)M * M);
    if (e != cudaSuccess) {
        cudaGetLastError();
        xcf_library_free(lib);
        return fail(ctx, XCF_ERR_OOM, "xcf_build_library: allocation failed");
    }
    e = cudaMemcpyAsync(lib->quats, quats, sizeof(double) * 4 * T, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lib->master, master, sizeof(float) * 2 * (size_t)M * M, cudaMemcpyDeviceToDevice, st);
    // project and pre-process in chunks (bounded image scratch)
    const ProjArgs pj = proj_args_cropped(g, c, ctx->opt.master_interp);
    const PrepArgs ps = prep_args_square(c, r);
    int *degen = nullptr;
    float *img = nullptr;
    for (int t0 = 0; spectra && e == cudaSuccess && t0 < T; t0 += kChunk) {
        const int nt = T - t0 < kChunk ? T - t0 : kChunk;
        if ((rc = scratch_t(ctx, S_IMG, (size_t)nt * c.n * c.n, &img)) ||
            (rc = scratch_t(ctx, S_DEGEN, nt, &degen))) {
            xcf_library_free(lib);
            return rc;
        }
        if (fused_project_prep(c.n)) {   // projected and pre-processed in one kernel
            ProjSrc src;
            src.master = lib->master;
            src.M = M;
            src.quats = lib->quats + 4 * (size_t)t0;
            src.a = pj;
            e = launch_prep_projected(src, nt, ps, lib->spectra + H * t0, nullptr, degen, nullptr, st);
        } else {
            e = launch_project(lib->master, M, lib->quats + 4 * (size_t)t0, nullptr, nullptr, nt, pj, img, st);
            if (e == cudaSuccess) e = run_prep(ctx, img, nt, ps, lib->spectra + H * t0, nullptr, degen, nullptr, st);
            ctx->launches[XCF_STAGE_PROJECT] += 1;
        }
        ctx->launches[XCF_STAGE_PREP] += 1;
    }
    if (spectra && e == cudaSuccess && has_search_layout(c.n)) {
        e = cudaMalloc(&lib->spectra_pk, sizeof(float2) * search_layout_f2(c.n) * T);
        if (e == cudaSuccess) e = launch_pack_search_layout(lib->spectra, T, c.n, lib->spectra_pk, st);
        ctx->launches[XCF_STAGE_OTHER] += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        xcf_library_free(lib);
        return cuda_fail(ctx, e, "xcf_build_library");
    }
    *out = lib;
    return XCF_OK;
}

int build_from_images(xcf_ctx *ctx, const float *images, const double *quats, int32_t T, const xcf_geometry *g,
                      const float *master, int32_t M, bool spectra, xcf_library **out, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!images || !quats || !g || !out || T <= 0 || (master && M < 2))
        return fail(ctx, XCF_ERR_ARG, "xcf_build_library_images: bad argument");
    *out = nullptr;
    Crop c;
    int rc = crop_of(g, 256, &c, ctx->opt.native_sizes != 0);
    if (rc) return fail(ctx, rc, "xcf_build_library_images: detector too small");
    if (!supported_n(c.n)) return fail(ctx, XCF_ERR_UNIMPLEMENTED, "xcf_build_library_images: detector side not supported");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Resolved r = resolve(ctx->opt, c.n);
    xcf_library *lib = new xcf_library();
    lib->device = ctx->device;
    lib->T = T;
    lib->N = c.n;
    lib->native = ctx->opt.native_sizes != 0;
    lib->M = master ? M : 0;
    lib->geom = *g;
    lib->ox = c.ox;
    lib->oy = c.oy;
    memcpy(lib->pc, c.pc, sizeof c.pc);
    const size_t H = (size_t)c.n * (c.n / 2 + 1);
    cudaError_t e = spectra ? cudaMalloc(&lib->spectra, sizeof(float2) * H * T) : cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&lib->quats, sizeof(double) * 4 * T);
    if (e == cudaSuccess && master) e = cudaMalloc(&lib->master, sizeof(float) * 2 * (size_t)M * M);
    if (e != cudaSuccess) {
        cudaGetLastError();
        xcf_library_free(lib);
        return fail(ctx, XCF_ERR_OOM, "xcf_build_library_images: allocation failed");
    }
    e = cudaMemcpyAsync(lib->quats, quats, sizeof(double) * 4 * T, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && master)
        e = cudaMemcpyAsync(lib->master, master, sizeof(float) * 2 * (size_t)M * M, cudaMemcpyDeviceToDevice, st);
    int *degen = nullptr;
    if ((rc = scratch_t(ctx, S_DEGEN, T, &degen))) {
        xcf_library_free(lib);
        return rc;
    }
    if (spectra) {
        if (e == cudaSuccess)
            e = run_prep(ctx, images, T, prep_args(g, c, r), lib->spectra, nullptr, degen, nullptr, st);
        ctx->launches[XCF_STAGE_PREP] += 1;
    }
    if (spectra && e == cudaSuccess && has_search_layout(c.n)) {
        e = cudaMalloc(&lib->spectra_pk, sizeof(float2) * search_layout_f2(c.n) * T);
        if (e == cudaSuccess) e = launch_pack_search_layout(lib->spectra, T, c.n, lib->spectra_pk, st);
        ctx->launches[XCF_STAGE_OTHER] += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        xcf_library_free(lib);
        return cuda_fail(ctx, e, "xcf_build_library_images");
    }
    *out = lib;
    return XCF_OK;
}
}  // namespace

int xcf_library_free(xcf_library *lib) {
    if (!lib) return XCF_ERR_ARG;
    cudaSetDevice(lib->device);
    if (lib->spectra) cudaFree(lib->spectra);
    if (lib->spectra_pk) cudaFree(lib->spectra_pk);
    if (lib->bf16) cudaFree(lib->bf16);
    if (lib->ndp32) cudaFree(lib->ndp32);
    if (lib->quats) cudaFree(lib->quats);
    if (lib->master) cudaFree(lib->master);
    delete lib;
    return XCF_OK;
}

int xcf_library_info(const xcf_library *lib, int32_t *T, int32_t *N, const float **spectra) {
    if (!lib) return XCF_ERR_ARG;
    if (T) *T = lib->T;
    if (N) *N = lib->N;
    if (spectra) *spectra = reinterpret_cast<const float *>(lib->spectra);
    return XCF_OK;
}

int xcf_index(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const double *pcs,
              int32_t *best, float *peak, float *shift, void *stream) {
    int rc = check_lib(ctx, lib, true);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !peak || !shift || P < 0) return fail(ctx, XCF_ERR_ARG, "xcf_index: bad argument");
    cudaSetDevice(ctx->device);
    const size_t img = (size_t)lib->geom.width * lib->geom.height;
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        if ((rc = index_chunk(ctx, lib, patterns + img * p0, np, best + p0, peak + p0, shift + 2 * (size_t)p0,
                              nullptr, (cudaStream_t)stream, nullptr, pcs ? pcs + 3 * (size_t)p0 : nullptr)))
            return rc;
    }
    return XCF_OK;
}

int xcf_correlate_all(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, float *peaks,
                      void *stream) {
    int rc = check_lib(ctx, lib, true);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !peaks || P < 0) return fail(ctx, XCF_ERR_ARG, "xcf_correlate_all: bad argument");
    cudaSetDevice(ctx->device);
    const size_t img = (size_t)lib->geom.width * lib->geom.height;
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        if ((rc = index_chunk(ctx, lib, patterns + img * p0, np, nullptr, nullptr, nullptr,
                              peaks + (size_t)lib->T * p0, (cudaStream_t)stream)))
            return rc;
    }
    return XCF_OK;
}

int xcf_refine(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const double *seeds,
               const double *pcs, int32_t max_iter, double tol_deg, double *quats, float *peak, int32_t *iters,
               void *stream) {
    int rc = check_lib(ctx, lib);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !seeds || !quats || !peak || !iters || P < 0)
        return fail(ctx, XCF_ERR_ARG, "xcf_refine: bad argument");
    if (!lib->master) return fail(ctx, XCF_ERR_ARG, "xcf_refine: library has no master pattern");
    if (max_iter > 1000) return fail(ctx, XCF_ERR_ARG, "xcf_refine: max_iter above 1000");
    const Resolved r = resolve(ctx->opt, lib->N);
    if (r.neta < 8 || r.neta > 1024 || (r.neta & (r.neta - 1)) || r.nr < 1 || r.rmin <= 0 ||
        r.rmax <= r.rmin || r.rmax > lib->N / 2.0 - 1.0)
        return fail(ctx, XCF_ERR_ARG, "xcf_refine: log-polar options out of range");
    cudaSetDevice(ctx->device);
    const size_t img = (size_t)lib->geom.width * lib->geom.height;
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        if ((rc = refine_chunk(ctx, lib, patterns + img * p0, np, seeds + 4 * (size_t)p0,
                               pcs ? pcs + 3 * (size_t)p0 : nullptr, quats + 4 * (size_t)p0, peak + p0,
                               iters + p0, (cudaStream_t)stream, nullptr, false, max_iter, tol_deg)))
            return rc;
    }
    return XCF_OK;
}

int xcf_disorientation(xcf_ctx *ctx, const double *qa, const double *qb, int32_t n, double *out, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (n == 0) return XCF_OK;
    if (!qa || !qb || !out || n < 0) return fail(ctx, XCF_ERR_ARG, "xcf_disorientation: bad argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_disorientation(qa, qb, n, out, st), "disorientation");
    return XCF_OK;
}

int xcf_index_refine(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const double *pcs,
                     int32_t *best, float *peak, float *shift, double *quats, float *rpeak, int32_t *iters,
                     void *stream) {
    int rc = check_lib(ctx, lib, true);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !peak || !shift || !quats || !rpeak || !iters || P < 0)
        return fail(ctx, XCF_ERR_ARG, "xcf_index_refine: bad argument");
    if (!lib->master) return fail(ctx, XCF_ERR_ARG, "xcf_index_refine: library has no master pattern");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t img = (size_t)lib->geom.width * lib->geom.height;
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        double *seeds;
        if ((rc = index_chunk(ctx, lib, patterns + img * p0, np, best + p0, peak + p0, shift + 2 * (size_t)p0,
                              nullptr, st, nullptr, pcs ? pcs + 3 * (size_t)p0 : nullptr)))
            return rc;
        if ((rc = scratch_t(ctx, S_SEEDS, (size_t)np * 4, &seeds))) return rc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_gather_seeds(lib->quats, best + p0, np, seeds, st), "seeds");
        if ((rc = refine_chunk(ctx, lib, patterns + img * p0, np, seeds, pcs ? pcs + 3 * (size_t)p0 : nullptr,
                               quats + 4 * (size_t)p0, rpeak + p0, iters + p0, st)))
            return rc;
    }
    return XCF_OK;
}

int xcf_refine_best(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const int32_t *best,
                    const double *pcs, double *quats, float *peak, int32_t *iters, void *stream) {
    int rc = check_lib(ctx, lib);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !quats || !peak || !iters || P < 0)
        return fail(ctx, XCF_ERR_ARG, "xcf_refine_best: bad argument");
    if (!lib->master) return fail(ctx, XCF_ERR_ARG, "xcf_refine_best: library has no master pattern");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t img = (size_t)lib->geom.width * lib->geom.height;
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        double *seeds;
        if ((rc = scratch_t(ctx, S_SEEDS, (size_t)np * 4, &seeds))) return rc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_gather_seeds(lib->quats, best + p0, np, seeds, st), "seeds");
        if ((rc = refine_chunk(ctx, lib, patterns + img * p0, np, seeds, pcs ? pcs + 3 * (size_t)p0 : nullptr,
                               quats + 4 * (size_t)p0, peak + p0, iters + p0, st)))
            return rc;
    }
    return XCF_OK;
}

int xcf_index_refine_host(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                          const double *pcs, int32_t chunk, int32_t *best, float *peak, float *shift,
                          double *quats, float *rpeak, int32_t *iters) {
    int rc = check_lib(ctx, lib, true);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !peak || !shift || !quats || !rpeak || !iters || P < 0)
        return fail(ctx, XCF_ERR_ARG, "xcf_index_refine_host: bad argument");
    if (chunk <= 0) {   // about four chunks (at least 2,048 patterns each), so that copies overlap compute
        chunk = (P + 3) / 4;
        if (chunk < 2048) chunk = 2048;
    }
    if (chunk > kChunk) chunk = kChunk;
    if (chunk > P) chunk = P;
    cudaSetDevice(ctx->device);
    const size_t img = (size_t)lib->geom.width * lib->geom.height;
    // two device slots of one chunk each: patterns | pcs | outputs; chunk i uses slot i & 1.
    // The copy stream moves chunk i + 1 in while the compute stream works on chunk i.
    float *dpat;
    double *dpcs = nullptr, *dseeds;
    const size_t out_bytes = ((size_t)chunk * (4 + 4 + 8 + 32 + 4 + 4) + 255) & ~(size_t)255;
    char *dout;
    if ((rc = scratch_t(ctx, S_IO_PAT, 2 * img * chunk, &dpat)) ||
        (pcs && (rc = scratch_t(ctx, S_IO_PCS, (size_t)2 * chunk * 3, &dpcs))) ||
        (rc = scratch_t(ctx, S_IO_OUT, 2 * out_bytes, &dout)) ||
        (rc = scratch_t(ctx, S_SEEDS, (size_t)chunk * 4, &dseeds)))
        return rc;
    cudaStream_t cs = nullptr, xs = nullptr;   // compute, copies
    cudaEvent_t ev[8] = {};                    // per slot: in_ready, in_free, out_ready, out_free
    int status = XCF_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) status = cuda_fail(ctx, e, "xcf_index_refine_host: streams");
    auto slot_out = [&](int sl, double **q, int **b, int **it, float **pk, float **sh, float **rp) {
        char *o = dout + sl * out_bytes;
        *q = reinterpret_cast<double *>(o);
        *b = reinterpret_cast<int *>(*q + 4 * (size_t)chunk);
        *it = *b + chunk;
        *pk = reinterpret_cast<float *>(*it + chunk);
        *sh = *pk + chunk;
        *rp = *sh + 2 * (size_t)chunk;
    };
    auto h2d = [&](int c) -> cudaError_t {   // chunk c in, on the copy stream
        const int sl = c & 1, p0 = c * chunk, np = P - p0 < chunk ? P - p0 : chunk;
        cudaError_t r = c >= 2 ? cudaStreamWaitEvent(xs, ev[4 * sl + 1], 0) : cudaSuccess;   // slot read by c - 2
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(dpat + img * chunk * sl, patterns + img * p0, sizeof(float) * img * np,
                                cudaMemcpyHostToDevice, xs);
        if (r == cudaSuccess && pcs)
            r = cudaMemcpyAsync(dpcs + (size_t)3 * chunk * sl, pcs + 3 * (size_t)p0, sizeof(double) * 3 * np,
                                cudaMemcpyHostToDevice, xs);
        if (r == cudaSuccess) r = cudaEventRecord(ev[4 * sl], xs);
        return r;
    };
    const int nchunks = (P + chunk - 1) / chunk;
    if (status == XCF_OK && (e = h2d(0)) != cudaSuccess) status = cuda_fail(ctx, e, "H2D");
    for (int c = 0; c < nchunks && status == XCF_OK; ++c) {
        const int sl = c & 1, p0 = c * chunk, np = P - p0 < chunk ? P - p0 : chunk;
        if (c + 1 < nchunks && (e = h2d(c + 1)) != cudaSuccess) { status = cuda_fail(ctx, e, "H2D"); break; }
        double *dq;
        int *dbest, *diters;
        float *dpeak, *dshift, *drpeak;
        slot_out(sl, &dq, &dbest, &diters, &dpeak, &dshift, &drpeak);
        const float *pat = dpat + img * chunk * sl;
        const double *pc = pcs ? dpcs + (size_t)3 * chunk * sl : nullptr;
        e = cudaStreamWaitEvent(cs, ev[4 * sl], 0);                      // chunk c is in
        if (e == cudaSuccess && c >= 2) e = cudaStreamWaitEvent(cs, ev[4 * sl + 3], 0);   // outputs of c - 2 read
        if (e != cudaSuccess) { status = cuda_fail(ctx, e, "wait"); break; }
        if ((status = index_chunk(ctx, lib, pat, np, dbest, dpeak, dshift, nullptr, cs, nullptr, pc))) break;
        e = launch_gather_seeds(lib->quats, dbest, np, dseeds, cs);
        if (e != cudaSuccess) { status = cuda_fail(ctx, e, "seeds"); break; }
        ctx->launches[XCF_STAGE_OTHER] += 1;
        if ((status = refine_chunk(ctx, lib, pat, np, dseeds, pc, dq, drpeak, diters, cs))) break;
        e = cudaEventRecord(ev[4 * sl + 1], cs);                         // slot's inputs no longer read
        if (e == cudaSuccess) e = cudaEventRecord(ev[4 * sl + 2], cs);   // outputs ready
        if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, ev[4 * sl + 2], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(best + p0, dbest, sizeof(int) * np, cudaMemcpyDeviceToHost, xs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(peak + p0, dpeak, sizeof(float) * np, cudaMemcpyDeviceToHost, xs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(shift + 2 * (size_t)p0, dshift, sizeof(float) * 2 * np, cudaMemcpyDeviceToHost, xs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(quats + 4 * (size_t)p0, dq, sizeof(double) * 4 * np, cudaMemcpyDeviceToHost, xs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rpeak + p0, drpeak, sizeof(float) * np, cudaMemcpyDeviceToHost, xs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(iters + p0, diters, sizeof(int) * np, cudaMemcpyDeviceToHost, xs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[4 * sl + 3], xs);   // outputs read
        if (e != cudaSuccess) status = cuda_fail(ctx, e, "D2H");
    }
    if (cs) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess && status == XCF_OK) status = cuda_fail(ctx, e, "xcf_index_refine_host");
    }
    if (xs) {
        e = cudaStreamSynchronize(xs);
        if (e != cudaSuccess && status == XCF_OK) status = cuda_fail(ctx, e, "xcf_index_refine_host");
    }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (xs) cudaStreamDestroy(xs);
    if (cs) cudaStreamDestroy(cs);
    return status;
}

int xcf_fp32_fma_rate(xcf_ctx *ctx, double *tflops, double *ms, void *stream) {
    if (!ctx || !tflops) return XCF_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    float *sink;
    int rc;
    if ((rc = scratch_t(ctx, S_PROBE, 1, &sink))) return rc;
    const int threads = 1024, blocks = 4 * ctx->num_sms, iters = 4096;
    cudaEvent_t a = nullptr, b = nullptr;
    XCF_CHECK(cudaEventCreate(&a), "event");
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(ctx, XCF_ERR_CUDA, "xcf_fp32_fma_rate: event");
    }
    cudaError_t e = launch_fma_rate(blocks, threads, iters / 8, sink, st);   // warm-up
    float best = 0.f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        float t = 0.f;
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) e = launch_fma_rate(blocks, threads, iters, sink, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e == cudaSuccess && (best == 0.f || t < best)) best = t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "xcf_fp32_fma_rate");
    ctx->launches[XCF_STAGE_OTHER] += 4;
    *tflops = fma_rate_flops(blocks, threads, iters) / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return XCF_OK;
}

int xcf_set_scratch_limit(xcf_ctx *ctx, uint64_t bytes) {
    if (!ctx) return XCF_ERR_ARG;
    ctx->scratch_limit = (size_t)bytes;
    return XCF_OK;
}

int xcf_scratch_bytes(const xcf_ctx *ctx, uint64_t *bytes) {
    if (!ctx || !bytes) return XCF_ERR_ARG;
    uint64_t t = 0;
    for (int i = 0; i < S_COUNT; ++i) t += ctx->cap[i];
    *bytes = t;
    return XCF_OK;
}

int xcf_profile_enable(xcf_ctx *ctx, int on) {
    if (!ctx) return XCF_ERR_ARG;
    ctx->timing = on != 0;
    return XCF_OK;
}

int xcf_profile_read(xcf_ctx *ctx, double *ms, int64_t *launches, int reset) {
    if (!ctx) return XCF_ERR_ARG;
    cudaSetDevice(ctx->device);
    int status = XCF_OK;
    for (auto &r : ctx->recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && status == XCF_OK) status = cuda_fail(ctx, e, "xcf_profile_read");
        ctx->ms[r.stage] += t;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->recs.clear();
    for (int i = 0; i < XCF_NUM_STAGES; ++i) {
        if (ms) ms[i] = ctx->ms[i];
        if (launches) launches[i] = ctx->launches[i];
        if (reset) {
            ctx->ms[i] = 0.0;
            ctx->launches[i] = 0;
        }
    }
    return status;
}

// ---------------------------------------------------------------- screen
namespace {

// chunk of patterns/templates whose f32 images and scores stay within ~1 GB
int screen_chunk(int n, int T) {
    const size_t lim = (size_t)1 << 30;
    size_t c = lim / ((size_t)n * n * 4);
    const size_t c2 = lim / ((size_t)(T > 0 ? T : 1) * 4);
    if (c2 < c) c = c2;
    if (c > (size_t)kChunk) c = kChunk;
    return c < 1 ? 1 : (int)c;
}

// BF16 unit-norm filtered images of the library's templates: from the
// caller's template images, or re-projected from the master
int make_screen_images(xcf_ctx *ctx, xcf_library *lib, const float *images, cudaStream_t st) {
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const size_t nn = (size_t)c.n * c.n, H = (size_t)c.n * (c.n / 2 + 1);
    if (cudaMalloc(&lib->bf16, 2 * nn * lib->T) != cudaSuccess) {
        cudaGetLastError();
        lib->bf16 = nullptr;
        return fail(ctx, XCF_ERR_OOM, "screen images: allocation failed");
    }
    const int chunk = screen_chunk(c.n, 1);
    int rc;
    for (int t0 = 0; t0 < lib->T; t0 += chunk) {
        const int nt = lib->T - t0 < chunk ? lib->T - t0 : chunk;
        float2 *spec;
        float *spat, *img;
        int *degen;
        if ((rc = scratch_t(ctx, S_SPEC_T, H * nt, &spec)) || (rc = scratch_t(ctx, S_SPATIAL_T, nn * nt, &spat)) ||
            (rc = scratch_t(ctx, S_DEGEN, nt, &degen)))
            return rc;
        if (images) {
            XCF_LAUNCH(XCF_STAGE_PREP, st,
                       run_prep(ctx, images + (size_t)g->width * g->height * t0, nt, prep_args(g, c, r), spec, spat,
                                degen, nullptr, st),
                       "screen prep");
        } else {
            if ((rc = scratch_t(ctx, S_IMG, nn * nt, &img))) return rc;
            XCF_LAUNCH(XCF_STAGE_PROJECT, st,
                       launch_project(lib->master, lib->M, lib->quats + 4 * (size_t)t0, nullptr, nullptr, nt,
                                      proj_args_cropped(g, c, ctx->opt.master_interp), img, st),
                       "screen project");
            XCF_LAUNCH(XCF_STAGE_PREP, st,
                       run_prep(ctx, img, nt, prep_args_square(c, r), spec, spat, degen, nullptr, st), "screen prep");
        }
        XCF_LAUNCH(XCF_STAGE_OTHER, st,
                   launch_to_bf16(spat, nn * nt, static_cast<char *>(lib->bf16) + 2 * nn * t0, st), "bf16");
    }
    return XCF_OK;
}

// contrast-normalised FP32 and BF16 images of the library's templates (NDP,
// Eq. 1): from the caller's template images, or re-projected from the master
int make_ndp_images(xcf_ctx *ctx, xcf_library *lib, const float *images, cudaStream_t st) {
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const size_t nn = (size_t)c.n * c.n;
    void *mem = nullptr;
    if (cudaMalloc(&mem, 6 * nn * lib->T) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, XCF_ERR_OOM, "NDP images: allocation failed");
    }
    lib->ndp32 = static_cast<float *>(mem);
    lib->ndp16 = static_cast<char *>(mem) + 4 * nn * lib->T;
    const int chunk = screen_chunk(c.n, 1);
    int rc;
    for (int t0 = 0; t0 < lib->T; t0 += chunk) {
        const int nt = lib->T - t0 < chunk ? lib->T - t0 : chunk;
        float *o32 = lib->ndp32 + nn * t0;
        void *o16 = static_cast<char *>(lib->ndp16) + 2 * nn * t0;
        if (images) {
            if ((rc = ndp_operands(ctx, images + (size_t)g->width * g->height * t0, nt, (long)g->width * g->height,
                                   g->width, c.ox, c.oy, c.n, o32, o16, nullptr, st)))
                return rc;
        } else {
            float *img;
            if ((rc = scratch_t(ctx, S_IMG, nn * nt, &img))) return rc;
            XCF_LAUNCH(XCF_STAGE_PROJECT, st,
                       launch_project(lib->master, lib->M, lib->quats + 4 * (size_t)t0, nullptr, nullptr, nt,
                                      proj_args_cropped(g, c, ctx->opt.master_interp), img, st),
                       "ndp project");
            if ((rc = ndp_operands(ctx, img, nt, (long)nn, c.n, 0, 0, c.n, o32, o16, nullptr, st))) return rc;
        }
    }
    return XCF_OK;
}

}  // namespace

int xcf_build_library_ex(xcf_ctx *ctx, const float *master, int32_t M, const double *quats, int32_t T,
                         const xcf_geometry *g, const float *images, int32_t flags, xcf_library **out,
                         void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!out) return fail(ctx, XCF_ERR_ARG, "xcf_build_library_ex: out is NULL");
    if (flags & ~(XCF_LIB_SCREEN | XCF_LIB_NDP | XCF_LIB_NO_SPECTRA))
        return fail(ctx, XCF_ERR_ARG, "xcf_build_library_ex: unknown flags");
    const bool spectra = !(flags & XCF_LIB_NO_SPECTRA);
    int rc = images ? build_from_images(ctx, images, quats, T, g, master, M, spectra, out, stream)
                    : build_from_master(ctx, master, M, quats, T, g, spectra, out, stream);
    if (rc || !(flags & (XCF_LIB_SCREEN | XCF_LIB_NDP))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (flags & XCF_LIB_SCREEN) rc = make_screen_images(ctx, *out, images, st);
    if (rc == XCF_OK && (flags & XCF_LIB_NDP)) rc = make_ndp_images(ctx, *out, images, st);
    if (rc == XCF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = cuda_fail(ctx, cudaGetLastError(), "screen images");
    if (rc) {
        xcf_library_free(*out);
        *out = nullptr;
    }
    return rc;
}

int xcf_screen_topk(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, int32_t k,
                    int32_t *cand, float *score, void *stream) {
    int rc = check_lib(ctx, lib);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !cand || !score || P < 0 || k < 1 || k > 64)
        return fail(ctx, XCF_ERR_ARG, "xcf_screen_topk: bad argument (1 <= k <= 64)");
    if (!lib->bf16) return fail(ctx, XCF_ERR_ARG, "xcf_screen_topk: library built without XCF_LIB_SCREEN");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const size_t nn = (size_t)c.n * c.n, H = (size_t)c.n * (c.n / 2 + 1), img = (size_t)g->width * g->height;
    if ((size_t)lib->T * 4 > 200 * 1024) return fail(ctx, XCF_ERR_SIZE, "xcf_screen_topk: more than 51,200 templates");
    const int chunk = screen_chunk(c.n, lib->T);
    int *err;
    if ((rc = scratch_t(ctx, S_ERR, 1, &err))) return rc;
    XCF_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st), "clear status");
    for (int p0 = 0; p0 < P; p0 += chunk) {
        const int np = P - p0 < chunk ? P - p0 : chunk;
        float2 *spec;
        float *spat, *S;
        int *degen;
        void *a;
        if ((rc = scratch_t(ctx, S_SPEC_P, H * np, &spec)) || (rc = scratch_t(ctx, S_SPATIAL_P, nn * np, &spat)) ||
            (rc = scratch_t(ctx, S_DEGEN, np, &degen)) || (rc = scratch(ctx, S_BF16_P, 2 * nn * np, &a)) ||
            (rc = scratch_t(ctx, S_SCORE, (size_t)np * lib->T, &S)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_PREP, st,
                   run_prep(ctx, patterns + img * p0, np, prep_args(g, c, r), spec, spat, degen, nullptr, st),
                   "screen prep");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_to_bf16(spat, nn * np, a, st), "bf16");
        XCF_LAUNCH(XCF_STAGE_SCREEN, st, launch_screen_tc(a, np, lib->bf16, lib->T, (int)nn, S, err, st), "screen");
        XCF_LAUNCH(XCF_STAGE_OTHER, st,
                   launch_topk_rows(S, np, lib->T, k, cand + (size_t)k * p0, score + (size_t)k * p0, st), "topk");
    }
    int h_err = 0;
    XCF_CHECK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    XCF_CHECK(cudaStreamSynchronize(st), "xcf_screen_topk");
    if (h_err) return fail(ctx, XCF_ERR_TIMEOUT, "xcf_screen_topk: a tensor-core pipeline wait timed out");
    return XCF_OK;
}

int xcf_rescore(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, const int32_t *cand,
                int32_t k, int32_t *best, float *peak, float *shift, void *stream) {
    int rc = check_lib(ctx, lib, true);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !cand || !best || !peak || !shift || P < 0 || k < 1)
        return fail(ctx, XCF_ERR_ARG, "xcf_rescore: bad argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const size_t H = (size_t)c.n * (c.n / 2 + 1), img = (size_t)g->width * g->height;
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        float2 *sp;
        int *degen;
        unsigned long long *keys;
        if ((rc = scratch_t(ctx, S_SPEC_P, H * np, &sp)) || (rc = scratch_t(ctx, S_DEGEN, np, &degen)) ||
            (rc = scratch_t(ctx, S_KEYS, np, &keys)))
            return rc;
        const int *cp = cand + (size_t)k * p0;
        XCF_LAUNCH(XCF_STAGE_PREP, st,
                   run_prep(ctx, patterns + img * p0, np, prep_args(g, c, r), sp, nullptr, degen, nullptr, st),
                   "prep");
        XCF_CHECK(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * np, st), "memset keys");
        if (c.n != 256) {
            XCF_LAUNCH(XCF_STAGE_SEARCH, st,
                       launch_search_list(c.n, lib->spectra, cp, k, sp, degen, np, keys, nullptr, ctx->num_sms, st),
                       "rescore");
        } else {
            XCF_LAUNCH(XCF_STAGE_SEARCH, st,
                       launch_search_c256(search_spectra(lib), 0, sp, degen, np, keys, nullptr, cp, k, st), "rescore");
        }
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_keys_to_best(keys, np, best + p0, st), "keys_to_best");
        XCF_LAUNCH(XCF_STAGE_PEAK, st,
                   run_pair_peak(ctx, c.n, lib->spectra, best + p0, sp, degen, nullptr, np, peak + p0,
                                 shift + 2 * (size_t)p0, st),
                   "pair_peak");
    }
    return XCF_OK;
}

int xcf_index_precision(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                        const double *pcs, int32_t k, int32_t *best, double *quats, float *peak, int32_t *iters,
                        void *stream) {
    int rc = check_lib(ctx, lib, true);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !quats || !peak || !iters || P < 0 || k < 1 || k > 64)
        return fail(ctx, XCF_ERR_ARG, "xcf_index_precision: bad argument (1 <= k <= 64)");
    if (!lib->bf16) return fail(ctx, XCF_ERR_ARG, "xcf_index_precision: library built without XCF_LIB_SCREEN");
    if (!lib->master) return fail(ctx, XCF_ERR_ARG, "xcf_index_precision: library has no master pattern");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const size_t nn = (size_t)c.n * c.n, H = (size_t)c.n * (c.n / 2 + 1), img = (size_t)g->width * g->height;
    if ((size_t)lib->T * 4 > 200 * 1024)
        return fail(ctx, XCF_ERR_SIZE, "xcf_index_precision: more than 51,200 templates");
    const int chunk = screen_chunk(c.n, lib->T);
    int *err;
    if ((rc = scratch_t(ctx, S_ERR, 1, &err))) return rc;
    XCF_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st), "clear status");
    for (int p0 = 0; p0 < P; p0 += chunk) {
        const int np = P - p0 < chunk ? P - p0 : chunk;
        const float *pat = patterns + img * p0;
        float2 *spec;
        float *spat, *S, *score;
        int *degen, *cand;
        unsigned long long *keys;
        double *seeds;
        void *a;
        if ((rc = scratch_t(ctx, S_SPEC_P, H * np, &spec)) || (rc = scratch_t(ctx, S_SPATIAL_P, nn * np, &spat)) ||
            (rc = scratch_t(ctx, S_DEGEN, np, &degen)) || (rc = scratch(ctx, S_BF16_P, 2 * nn * np, &a)) ||
            (rc = scratch_t(ctx, S_SCORE, (size_t)np * lib->T, &S)) || (rc = scratch_t(ctx, S_KEYS, np, &keys)) ||
            (rc = scratch_t(ctx, S_CAND, (size_t)np * k, &cand)) ||
            (rc = scratch_t(ctx, S_CANDSC, (size_t)np * k, &score)) ||
            (rc = scratch_t(ctx, S_SEEDS, (size_t)np * 4, &seeds)))
            return rc;
        // one pre-processing of the patterns serves the screen, the rescore and the refinement
        XCF_LAUNCH(XCF_STAGE_PREP, st, run_prep(ctx, pat, np, prep_args(g, c, r), spec, spat, degen, nullptr, st),
                   "prep");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_to_bf16(spat, nn * np, a, st), "bf16");
        XCF_LAUNCH(XCF_STAGE_SCREEN, st, launch_screen_tc(a, np, lib->bf16, lib->T, (int)nn, S, err, st), "screen");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_topk_rows(S, np, lib->T, k, cand, score, st), "topk");
        XCF_CHECK(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * np, st), "memset keys");
        if (c.n != 256) {
            XCF_LAUNCH(XCF_STAGE_SEARCH, st,
                       launch_search_list(c.n, lib->spectra, cand, k, spec, degen, np, keys, nullptr, ctx->num_sms,
                                          st),
                       "rescore");
        } else {
            XCF_LAUNCH(XCF_STAGE_SEARCH, st,
                       launch_search_c256(search_spectra(lib), 0, spec, degen, np, keys, nullptr, cand, k, st), "rescore");
        }
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_keys_to_best(keys, np, best + p0, st), "keys_to_best");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_gather_seeds(lib->quats, best + p0, np, seeds, st), "seeds");
        if ((rc = refine_chunk(ctx, lib, pat, np, seeds, pcs ? pcs + 3 * (size_t)p0 : nullptr, quats + 4 * (size_t)p0,
                               peak + p0, iters + p0, st, nullptr, true)))
            return rc;
    }
    int h_err = 0;
    XCF_CHECK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    XCF_CHECK(cudaStreamSynchronize(st), "xcf_index_precision");
    if (h_err) return fail(ctx, XCF_ERR_TIMEOUT, "xcf_index_precision: a tensor-core pipeline wait timed out");
    return XCF_OK;
}

// ------------------------------------------------------------------- NDP
int xcf_index_ndp(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P, int32_t k,
                  int32_t *best, float *ndp, int32_t *cand, float *cand_score, void *stream) {
    int rc = check_lib(ctx, lib);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !ndp || P < 0 || k < 1 || k > 64 || (!cand) != (!cand_score))
        return fail(ctx, XCF_ERR_ARG, "xcf_index_ndp: bad argument (1 <= k <= 64; cand and cand_score together)");
    if (!lib->ndp32) return fail(ctx, XCF_ERR_ARG, "xcf_index_ndp: library built without XCF_LIB_NDP");
    if ((size_t)lib->T * 4 > 200 * 1024) return fail(ctx, XCF_ERR_SIZE, "xcf_index_ndp: more than 51,200 templates");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const size_t nn = (size_t)c.n * c.n, img = (size_t)g->width * g->height;
    const int chunk = screen_chunk(c.n, lib->T);
    int *err;
    if ((rc = scratch_t(ctx, S_ERR, 1, &err))) return rc;
    XCF_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st), "clear status");
    for (int p0 = 0; p0 < P; p0 += chunk) {
        const int np = P - p0 < chunk ? P - p0 : chunk;
        float *pn, *S, *csc;
        int *degen, *cd;
        void *a;
        if ((rc = scratch_t(ctx, S_SPATIAL_P, nn * np, &pn)) || (rc = scratch_t(ctx, S_DEGEN, np, &degen)) ||
            (rc = scratch(ctx, S_BF16_P, 2 * nn * np, &a)) ||
            (rc = scratch_t(ctx, S_SCORE, (size_t)np * lib->T, &S)))
            return rc;
        if (cand) {
            cd = cand + (size_t)k * p0;
            csc = cand_score + (size_t)k * p0;
        } else if ((rc = scratch_t(ctx, S_CAND, (size_t)np * k, &cd)) ||
                   (rc = scratch_t(ctx, S_CANDSC, (size_t)np * k, &csc))) {
            return rc;
        }
        if ((rc = ndp_operands(ctx, patterns + img * p0, np, (long)img, g->width, c.ox, c.oy, c.n, pn, a, degen, st)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_SCREEN, st, launch_screen_tc(a, np, lib->ndp16, lib->T, (int)nn, S, err, st), "ndp gemm");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_topk_rows(S, np, lib->T, k, cd, csc, st), "topk");
        XCF_LAUNCH(XCF_STAGE_SEARCH, st,
                   launch_ndp_rescore(pn, lib->ndp32, (long)nn, cd, k, degen, np, best + p0, ndp + p0, st),
                   "ndp rescore");
    }
    int h_err = 0;
    XCF_CHECK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    XCF_CHECK(cudaStreamSynchronize(st), "xcf_index_ndp");
    if (h_err) return fail(ctx, XCF_ERR_TIMEOUT, "xcf_index_ndp: a tensor-core pipeline wait timed out");
    return XCF_OK;
}

int xcf_rotation_scan(xcf_ctx *ctx, const float *master, int32_t M, const xcf_geometry *g, const double *q,
                      const double *pc_test, int32_t h, double step_deg, float *ndp, float *xcf, float *fwhm,
                      void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!master || !g || !q || !ndp || !xcf || M < 2 || h < 1 || h > 2048 || !(step_deg > 0.0))
        return fail(ctx, XCF_ERR_ARG, "xcf_rotation_scan: bad argument (1 <= h <= 2048, step_deg > 0)");
    Crop c;
    int rc = crop_of(g, 256, &c, ctx->opt.native_sizes != 0);
    if (rc) return fail(ctx, rc, "xcf_rotation_scan: detector too small");
    if (!supported_n(c.n)) return fail(ctx, XCF_ERR_UNIMPLEMENTED, "xcf_rotation_scan: detector side not supported");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Resolved r = resolve(ctx->opt, c.n);
    const int L = 2 * h + 1, n_img = 1 + 3 * L, nt = 3 * L;
    const size_t nn = (size_t)c.n * c.n, H = (size_t)c.n * (c.n / 2 + 1);
    double *qs, *pcs;
    float *imgs, *pn, *shift;
    float2 *spec;
    int *degen, *zeros, *junk_best;
    if ((rc = scratch_t(ctx, S_SEEDS, (size_t)n_img * 4, &qs)) || (rc = scratch_t(ctx, S_Q1, (size_t)n_img * 3, &pcs)) ||
        (rc = scratch_t(ctx, S_IMG, nn * n_img, &imgs)) || (rc = scratch_t(ctx, S_SPATIAL_P, nn * n_img, &pn)) ||
        (rc = scratch_t(ctx, S_SPEC_P, H * n_img, &spec)) || (rc = scratch_t(ctx, S_DEGEN, n_img, &degen)) ||
        (rc = scratch_t(ctx, S_CAND, nt, &zeros)) || (rc = scratch_t(ctx, S_BEST, nt, &junk_best)) ||
        (rc = scratch_t(ctx, S_SHIFT, 2 * (size_t)nt, &shift)))
        return rc;
    XCF_CHECK(cudaMemsetAsync(zeros, 0, sizeof(int) * nt, st), "clear template indices");
    XCF_LAUNCH(XCF_STAGE_OTHER, st,
               launch_scan_setup(q, pc_test, g->pcx, g->pcy, g->pcz, h, step_deg * kPi / 180.0, alpha_of(g), qs, pcs,
                                 st),
               "scan setup");
    XCF_LAUNCH(XCF_STAGE_PROJECT, st,
               launch_project(master, M, qs, pcs, nullptr, n_img, proj_args_cropped(g, c, ctx->opt.master_interp),
                              imgs, st),
               "scan project");
    // Eq. 1: every image normalised, then each test image against the reference (entry 0)
    if ((rc = ndp_operands(ctx, imgs, n_img, (long)nn, c.n, 0, 0, c.n, pn, nullptr, degen, st))) return rc;
    XCF_LAUNCH(XCF_STAGE_SEARCH, st,
               launch_ndp_rescore(pn + nn, pn, (long)nn, zeros, 1, degen + 1, nt, junk_best, ndp, st), "ndp pairs");
    // FFT XCF: the reference's spectrum as the template of every test image
    XCF_LAUNCH(XCF_STAGE_PREP, st,
               run_prep(ctx, imgs, n_img, prep_args_square(c, r), spec, nullptr, degen, nullptr, st), "scan prep");
    XCF_LAUNCH(XCF_STAGE_PEAK, st,
               run_pair_peak(ctx, c.n, spec, zeros, spec + H, degen + 1, nullptr, nt, xcf, shift, st), "scan peak");
    if (fwhm) XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_fwhm(ndp, xcf, 6, L, (float)step_deg, fwhm, st), "fwhm");
    return XCF_OK;
}

// --------------------------------------------------------- SO(3) sampling
int xcf_nearest_disorientation(xcf_ctx *ctx, const double *qa, int32_t na, const double *qb, int32_t nb,
                               int32_t mode, double *angle_deg, int32_t *index, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (na == 0) return XCF_OK;
    if (!qb) {
        qb = qa;
        nb = na;
    }
    if (!qa || !angle_deg || !index || na < 0 || nb < 0 || mode < 0 || mode > 2 || (mode && qb != qa))
        return fail(ctx, XCF_ERR_ARG, "xcf_nearest_disorientation: bad argument (modes 1, 2 need qb == qa or NULL)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *keys;
    int rc;
    if ((rc = scratch_t(ctx, S_NN_KEYS, na, &keys))) return rc;
    XCF_LAUNCH(XCF_STAGE_OTHER, st,
               launch_nearest_disorientation(qa, na, qb, nb, mode, keys, angle_deg, index, ctx->num_sms, st),
               "nearest disorientation");
    return XCF_OK;
}

int xcf_so3_grid(xcf_ctx *ctx, double step_deg, int32_t flags, double *quats, int64_t cap, int64_t *count,
                 void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!count || !(step_deg >= 0.5 && step_deg <= 180.0) || (flags & ~XCF_SO3_DEDUP) || cap < 0)
        return fail(ctx, XCF_ERR_ARG, "xcf_so3_grid: bad argument (0.5 <= step_deg <= 180)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // ring sizes: integer bookkeeping of the scheme (sizes of the launches below)
    const double d = step_deg * kPi / 180.0;
    const long n_polar = std::max(1L, lround(kPi / d)), n_s1 = std::max(1L, lround(2 * kPi / d));
    const int n_rings = (int)n_polar + 1;
    std::vector<long long> start(n_rings);
    std::vector<int> az(n_rings);
    long long G = 0;
    for (int i = 0; i < n_rings; ++i) {
        az[i] = (int)std::max(1L, lround(2 * kPi * sin(kPi * i / n_polar) / d));
        start[i] = G;
        G += (long long)az[i] * n_s1;
    }
    long long *ring_start, *total;
    int *ring_az, *flag, *bc;
    double *q_all, *q_fz;
    int rc;
    const int nb = compact_blocks(G);
    if ((rc = scratch(ctx, S_SO3_RING, (sizeof(long long) + sizeof(int)) * n_rings, (void **)&ring_start)) ||
        (rc = scratch_t(ctx, S_SO3_QALL, 4 * (size_t)G, &q_all)) || (rc = scratch_t(ctx, S_SO3_FLAG, (size_t)G, &flag)) ||
        (rc = scratch(ctx, S_SO3_CNT, sizeof(long long) + sizeof(int) * (size_t)nb, (void **)&total)))
        return rc;
    ring_az = reinterpret_cast<int *>(ring_start + n_rings);
    bc = reinterpret_cast<int *>(total + 1);
    XCF_CHECK(cudaMemcpyAsync(ring_start, start.data(), sizeof(long long) * n_rings, cudaMemcpyHostToDevice, st),
              "ring starts");
    XCF_CHECK(cudaMemcpyAsync(ring_az, az.data(), sizeof(int) * n_rings, cudaMemcpyHostToDevice, st), "ring sizes");
    XCF_LAUNCH(XCF_STAGE_OTHER, st,
               launch_so3_points(ring_start, n_rings, (int)n_polar, (int)n_s1, ring_az, G, q_all, flag, st),
               "so3 points");
    long long n_fz = 0;
    XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_compact(q_all, flag, G, bc, total, nullptr, st), "so3 count");
    XCF_CHECK(cudaMemcpyAsync(&n_fz, total, sizeof n_fz, cudaMemcpyDeviceToHost, st), "so3 count");
    XCF_CHECK(cudaStreamSynchronize(st), "xcf_so3_grid");
    if (n_fz > INT32_MAX) return fail(ctx, XCF_ERR_SIZE, "xcf_so3_grid: more than 2^31 orientations");
    if ((rc = scratch_t(ctx, S_SO3_QFZ, 4 * (size_t)n_fz, &q_fz))) return rc;
    XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_compact(q_all, flag, G, bc, total, q_fz, st), "so3 zone");
    long long n = n_fz;
    const double *src = q_fz;
    if (flags & XCF_SO3_DEDUP) {
        double *ang;
        int *idx;
        unsigned long long *keys;
        if ((rc = scratch_t(ctx, S_NN_ANG, (size_t)n_fz, &ang)) || (rc = scratch_t(ctx, S_NN_IDX, (size_t)n_fz, &idx)) ||
            (rc = scratch_t(ctx, S_NN_KEYS, (size_t)n_fz, &keys)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st,
                   launch_nearest_disorientation(q_fz, (int)n_fz, q_fz, (int)n_fz, 2, keys, ang, idx, ctx->num_sms,
                                                 st),
                   "so3 copies");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_keep_flags(ang, n_fz, 1e-3, flag, st), "so3 keep");
        XCF_LAUNCH(XCF_STAGE_OTHER, st,
                   launch_compact(q_fz, flag, n_fz, bc, total, quats && cap >= n_fz ? quats : nullptr, st),
                   "so3 dedup");
        XCF_CHECK(cudaMemcpyAsync(&n, total, sizeof n, cudaMemcpyDeviceToHost, st), "so3 count");
        XCF_CHECK(cudaStreamSynchronize(st), "xcf_so3_grid");
        src = nullptr;   // written by the compaction (when it fitted)
        if (quats && cap < n_fz && cap >= n) {
            // the output could not hold the pre-duplicate set: compact again into it
            XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_compact(q_fz, flag, n_fz, bc, total, quats, st), "so3 dedup");
        }
    }
    *count = n;
    if (!quats) return XCF_OK;
    if (cap < n) return fail(ctx, XCF_ERR_SIZE, "xcf_so3_grid: cap smaller than the orientation count");
    if (src) XCF_CHECK(cudaMemcpyAsync(quats, src, sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice, st), "so3 out");
    XCF_CHECK(cudaStreamSynchronize(st), "xcf_so3_grid");
    return XCF_OK;
}

// ------------------------------------------------------ proposal network
namespace {

constexpr int kNetChunk = 1024;   // patterns per network pass (bounds the activations)

int net_input(xcf_ctx *ctx, const float *images, const xcf_geometry *g, CnnInput *in) {
    if (!g) {
        *in = {images, (long)XCF_NET_SIDE * XCF_NET_SIDE, XCF_NET_SIDE, 0, 0};
        return XCF_OK;
    }
    Crop c;
    if (crop_of(g, XCF_NET_SIDE, &c) != XCF_OK || c.n != XCF_NET_SIDE)
        return fail(ctx, XCF_ERR_SIZE, "proposal network: the detector must be at least 128 x 128");
    *in = {images, (long)g->width * g->height, g->width, c.ox, c.oy};
    return XCF_OK;
}

int net_reserve(xcf_ctx *ctx, xcf_net *net, int B, bool backward) {
    const size_t a = cnn_act_floats(B, net->k);
    if (net->act_cap < a) {
        cudaFree(net->act);
        net->act = nullptr;
        net->act_cap = 0;
        if (cudaMalloc(&net->act, sizeof(float) * a) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, XCF_ERR_OOM, "proposal network activations");
        }
        net->act_cap = a;
    }
    const size_t gb = cnn_grad_floats(B, net->k);
    if (backward && net->gbuf_cap < gb) {
        cudaFree(net->gbuf);
        net->gbuf = nullptr;
        net->gbuf_cap = 0;
        if (cudaMalloc(&net->gbuf, sizeof(float) * gb) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, XCF_ERR_OOM, "proposal network gradient buffers");
        }
        net->gbuf_cap = gb;
    }
    return XCF_OK;
}

int check_net(xcf_ctx *ctx, const xcf_net *net) {
    if (!ctx) return XCF_ERR_ARG;
    if (!net) return fail(ctx, XCF_ERR_ARG, "network is NULL");
    if (net->device != ctx->device) return fail(ctx, XCF_ERR_ARG, "network and context on different devices");
    return XCF_OK;
}

// forward of B <= kNetChunk images (FP32, or the BF16 inference form); the
// outputs stay in net->act
int net_forward_chunk(xcf_ctx *ctx, xcf_net *net, const CnnInput &in, int B, cudaStream_t st) {
    int rc = net_reserve(ctx, net, B, false);
    if (rc) return rc;
    int nl = 0;
    if (net->bf16) {
        void *work;
        int *err;
        if ((rc = scratch(ctx, S_NET_BF16, cnn_bf16_work_bytes(B), &work)) || (rc = scratch_t(ctx, S_ERR, 1, &err)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_NET, st, launch_cnn_forward_bf16(net->params, net->k, in, B, net->act, work, err, ctx->num_sms, &nl, st),
                   "net forward (bf16)");
    } else {
        XCF_LAUNCH(XCF_STAGE_NET, st, launch_cnn_forward(net->params, net->k, in, B, net->act, &nl, st),
                   "net forward");
    }
    ctx->launches[XCF_STAGE_NET] += nl - 1;
    return XCF_OK;
}

// the BF16 form's tensor-core status word: cleared before a call's forward
// passes, read (waiting for the device) after them
int net_status_begin(xcf_ctx *ctx, const xcf_net *net, cudaStream_t st) {
    if (!net->bf16) return XCF_OK;
    int *err, rc;
    if ((rc = scratch_t(ctx, S_ERR, 1, &err))) return rc;
    XCF_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st), "clear status");
    return XCF_OK;
}
int net_status_end(xcf_ctx *ctx, const xcf_net *net, cudaStream_t st, const char *fn) {
    if (!net->bf16) return XCF_OK;
    int *err, rc, h = 0;
    if ((rc = scratch_t(ctx, S_ERR, 1, &err))) return rc;
    XCF_CHECK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    XCF_CHECK(cudaStreamSynchronize(st), fn);
    if (h) return fail(ctx, XCF_ERR_TIMEOUT, std::string(fn) + ": a tensor-core pipeline wait timed out");
    return XCF_OK;
}

CnnInput offset_input(const CnnInput &in, long b0) {
    CnnInput o = in;
    o.x = in.x + b0 * in.img_stride;
    return o;
}

// proposals of P patterns -> quats [P][k][4]
int propose_all(xcf_ctx *ctx, xcf_net *net, const CnnInput &in, int P, double *quats, cudaStream_t st) {
    int rc0 = net_status_begin(ctx, net, st);
    if (rc0) return rc0;
    for (int b0 = 0; b0 < P; b0 += kNetChunk) {
        const int nb = P - b0 < kNetChunk ? P - b0 : kNetChunk;
        int rc = net_forward_chunk(ctx, net, offset_input(in, b0), nb, st);
        if (rc) return rc;
        XCF_LAUNCH(XCF_STAGE_NET, st,
                   launch_cnn_proposals(cnn_output(net->act, nb, net->k), nb * net->k,
                                        quats + (size_t)b0 * net->k * 4, st),
                   "proposals");
    }
    return net_status_end(ctx, net, st, "proposals");
}

}  // namespace

int64_t xcf_net_num_params(int32_t k) { return k >= 1 && k <= 64 ? (int64_t)cnn_num_params(k) : -1; }

int xcf_net_create(xcf_ctx *ctx, int32_t k, const float *params, xcf_net **out) {
    if (!ctx) return XCF_ERR_ARG;
    if (!out || k < 1 || k > 64) return fail(ctx, XCF_ERR_ARG, "xcf_net_create: bad argument");
    cudaSetDevice(ctx->device);
    xcf_net *net = new xcf_net();
    net->device = ctx->device;
    net->k = k;
    net->n = cnn_num_params(k);
    float *base = nullptr;
    cudaError_t e = cudaMalloc(&base, sizeof(float) * 4 * (size_t)net->n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete net;
        return fail(ctx, XCF_ERR_OOM, "xcf_net_create: parameters");
    }
    net->params = base;
    net->grad = base + net->n;
    net->m = base + 2 * net->n;
    net->v = base + 3 * net->n;
    e = cudaMemset(base, 0, sizeof(float) * 4 * (size_t)net->n);
    if (e == cudaSuccess && params)
        e = cudaMemcpy(net->params, params, sizeof(float) * net->n, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(base);
        delete net;
        return cuda_fail(ctx, e, "xcf_net_create");
    }
    *out = net;
    return XCF_OK;
}

int xcf_net_free(xcf_net *net) {
    if (!net) return XCF_ERR_ARG;
    cudaSetDevice(net->device);
    cudaFree(net->params);
    cudaFree(net->act);
    cudaFree(net->gbuf);
    delete net;
    return XCF_OK;
}

int xcf_net_params(xcf_net *net, float **params, int64_t *n) {
    if (!net) return XCF_ERR_ARG;
    if (params) *params = net->params;
    if (n) *n = net->n;
    return XCF_OK;
}

int xcf_net_forward(xcf_ctx *ctx, xcf_net *net, const float *images, int32_t B, const xcf_geometry *g, float *out,
                    void *stream) {
    int rc = check_net(ctx, net);
    if (rc) return rc;
    if (B == 0) return XCF_OK;
    if (B < 0 || !images || !out) return fail(ctx, XCF_ERR_ARG, "xcf_net_forward: bad argument");
    CnnInput in;
    if ((rc = net_input(ctx, images, g, &in))) return rc;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = net_status_begin(ctx, net, st))) return rc;
    for (int b0 = 0; b0 < B; b0 += kNetChunk) {
        const int nb = B - b0 < kNetChunk ? B - b0 : kNetChunk;
        if ((rc = net_forward_chunk(ctx, net, offset_input(in, b0), nb, st))) return rc;
        XCF_CHECK(cudaMemcpyAsync(out + (size_t)b0 * 6 * net->k, cnn_output(net->act, nb, net->k),
                                  sizeof(float) * 6 * net->k * nb, cudaMemcpyDeviceToDevice, st),
                  "net outputs");
    }
    return net_status_end(ctx, net, st, "xcf_net_forward");
}

int xcf_net_set_bf16(xcf_net *net, int32_t on) {
    if (!net || (on != 0 && on != 1)) return XCF_ERR_ARG;
    net->bf16 = on;
    return XCF_OK;
}

int xcf_net_loss_grad(xcf_ctx *ctx, xcf_net *net, const float *images, int32_t B, const xcf_geometry *g,
                      const double *quats_gt, double *loss, float *grad, int32_t *winners, void *stream) {
    int rc = check_net(ctx, net);
    if (rc) return rc;
    if (B <= 0 || !images || !quats_gt || !loss) return fail(ctx, XCF_ERR_ARG, "xcf_net_loss_grad: bad argument");
    CnnInput in;
    if ((rc = net_input(ctx, images, g, &in))) return rc;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = net_reserve(ctx, net, B, true))) return rc;
    XCF_CHECK(cudaMemsetAsync(loss, 0, sizeof(double), st), "loss");
    int nl = 0;
    XCF_LAUNCH(XCF_STAGE_NET, st, launch_cnn_forward(net->params, net->k, in, B, net->act, &nl, st), "net forward");
    XCF_LAUNCH(XCF_STAGE_NET, st,
               launch_cnn_backward(net->params, net->k, in, B, net->act, net->gbuf, quats_gt, loss, winners,
                                   net->grad, ctx->num_sms, &nl, st),
               "net backward");
    ctx->launches[XCF_STAGE_NET] += nl - 2;
    if (grad)
        XCF_CHECK(cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->n, cudaMemcpyDeviceToDevice, st),
                  "gradient");
    return XCF_OK;
}

int xcf_net_adam(xcf_ctx *ctx, xcf_net *net, float lr, float beta1, float beta2, float eps, void *stream) {
    int rc = check_net(ctx, net);
    if (rc) return rc;
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(ctx, XCF_ERR_ARG, "xcf_net_adam: bad hyper-parameter");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    net->t += 1;
    XCF_LAUNCH(XCF_STAGE_NET, st,
               launch_adam(net->params, net->grad, net->m, net->v, net->n, lr, beta1, beta2, eps, net->t, st),
               "adam");
    return XCF_OK;
}

int xcf_propose(xcf_ctx *ctx, xcf_net *net, const float *patterns, int32_t P, const xcf_geometry *g, double *quats,
                void *stream) {
    int rc = check_net(ctx, net);
    if (rc) return rc;
    if (P == 0) return XCF_OK;
    if (P < 0 || !patterns || !quats) return fail(ctx, XCF_ERR_ARG, "xcf_propose: bad argument");
    CnnInput in;
    if ((rc = net_input(ctx, patterns, g, &in))) return rc;
    cudaSetDevice(ctx->device);
    return propose_all(ctx, net, in, P, quats, (cudaStream_t)stream);
}

int xcf_index_learned(xcf_ctx *ctx, xcf_net *net, const xcf_library *lib, const float *patterns, int32_t P,
                      const double *pcs, float tau, double *quats, float *peak, int32_t *iters, int32_t *fallback,
                      void *stream) {
    int rc = check_net(ctx, net);
    if (rc) return rc;
    if ((rc = check_lib(ctx, lib, true))) return rc;
    if (P == 0) return XCF_OK;
    if (P < 0 || !patterns || !quats || !peak || !iters || !fallback)
        return fail(ctx, XCF_ERR_ARG, "xcf_index_learned: bad argument");
    if (!lib->master) return fail(ctx, XCF_ERR_ARG, "xcf_index_learned: library has no master pattern");
    CnnInput in;
    if ((rc = net_input(ctx, patterns, &lib->geom, &in))) return rc;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const xcf_geometry *g = &lib->geom;
    Crop c;
    crop_of(g, 256, &c, lib->native);
    const Resolved r = resolve(ctx->opt, c.n);
    const int n = c.n, H = n * (n / 2 + 1), k = net->k;
    const size_t img = (size_t)g->width * g->height;
    const ProjArgs pj = proj_args_cropped(g, c, ctx->opt.master_interp);
    const PrepArgs pa = prep_args(g, c, r), ps = prep_args_square(c, r);
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int np = P - p0 < kChunk ? P - p0 : kChunk;
        const float *pat = patterns + img * p0;
        const double *pc = pcs ? pcs + 3 * (size_t)p0 : nullptr;
        double *q = quats + 4 * (size_t)p0;
        double *prop, *qh;
        float2 *sp, *stt;
        float *img_t, *peak_h, *shift, *best_peak, *yp;
        int *degen, *count;
        if ((rc = scratch_t(ctx, S_PROP, (size_t)np * k * 4, &prop)) || (rc = scratch_t(ctx, S_QH, (size_t)np * 4, &qh)) ||
            (rc = scratch_t(ctx, S_SPEC_P, (size_t)np * H, &sp)) || (rc = scratch_t(ctx, S_SPEC_T, (size_t)np * H, &stt)) ||
            (rc = scratch_t(ctx, S_SPATIAL_P, (size_t)np * n * n, &yp)) ||
            (rc = scratch_t(ctx, S_IMG, (size_t)np * n * n, &img_t)) || (rc = scratch_t(ctx, S_PEAK, np, &peak_h)) ||
            (rc = scratch_t(ctx, S_SHIFT, (size_t)np * 2, &shift)) || (rc = scratch_t(ctx, S_BESTPEAK, np, &best_peak)) ||
            (rc = scratch_t(ctx, S_DEGEN, np, &degen)) || (rc = scratch_t(ctx, S_FBCOUNT, 2, &count)))
            return rc;
        // 1. proposals
        if ((rc = propose_all(ctx, net, offset_input(in, p0), np, prop, st))) return rc;
        // 2. correlation score of every proposal, the best kept as the seed (the
        // patterns' spectra, filtered images and flags stay for the refinement)
        XCF_LAUNCH(XCF_STAGE_PREP, st, run_prep(ctx, pat, np, pa, sp, yp, degen, nullptr, st), "prep patterns");
        for (int h = 0; h < k; ++h) {
            XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_take_head(prop, np, k, h, qh, st), "take head");
            if ((rc = project_prep(ctx, lib->master, lib->M, qh, pc, nullptr, np, pj, ps, stt, nullptr, nullptr, img_t,
                                   st)))
                return rc;
            XCF_LAUNCH(XCF_STAGE_PEAK, st, run_pair_peak(ctx, n, stt, nullptr, sp, degen, nullptr, np, peak_h, shift, st),
                       "proposal peaks");
            XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_keep_best(peak_h, qh, np, h, best_peak, q, nullptr, st), "keep best");
        }
        // 3. refinement of the best proposal, on the patterns pre-processed above
        if ((rc = refine_chunk(ctx, lib, pat, np, q, pc, q, peak + p0, iters + p0, st, nullptr, true))) return rc;
        // 4. fallback where the refined peak stays below tau
        if ((rc = scratch_t(ctx, S_DEGEN, np, &degen))) return rc;   // the refinement's pattern flags
        int *fidx, *flag_c;
        if ((rc = scratch_t(ctx, S_FB_IDX, (size_t)np + 1, &fidx)) ||
            (rc = scratch_t(ctx, S_FB_FLAG, (size_t)np + 1, &flag_c)))
            return rc;
        XCF_CHECK(cudaMemsetAsync(count, 0, 2 * sizeof(int), st), "count");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_fallback_flags(peak + p0, degen, np, tau, fallback + p0, count, st),
                   "fallback flags");
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_fallback_list(fallback + p0, np, fidx, flag_c, count + 1, st),
                   "fallback list");
        int counts[2] = {0, 0};
        XCF_CHECK(cudaMemcpyAsync(counts, count, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "count");
        XCF_CHECK(cudaStreamSynchronize(st), "count");
        if (counts[0] == 0) continue;
        // the flagged patterns gathered (by pattern pairs) into a batch of their
        // own: the full search then spreads the library over the SMs for them
        // alone, and the refinement runs on them alone
        const int nc = 2 * counts[1];
        int *best_c, *it_c;
        float *pat_c, *pk_c;
        double *pc_c = nullptr, *q_c;
        if ((rc = scratch_t(ctx, S_FB_PAT, (size_t)nc * img, &pat_c)) || (rc = scratch_t(ctx, S_FB_BEST, nc, &best_c)) ||
            (rc = scratch_t(ctx, S_FB_IT, nc, &it_c)) || (rc = scratch_t(ctx, S_FB_PEAK, (size_t)nc * 4, &pk_c)) ||
            (rc = scratch_t(ctx, S_FB_Q, (size_t)nc * 8, &q_c)) ||
            (pc && (rc = scratch_t(ctx, S_FB_PC, (size_t)nc * 3, &pc_c))))
            return rc;
        double *seeds_c = q_c + 4 * (size_t)nc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_gather_rows(pat, img, fidx, nc, pat_c, st), "gather patterns");
        if (pc) XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_gather_rows(pc, 3, fidx, nc, pc_c, st), "gather pcs");
        if ((rc = index_chunk(ctx, lib, pat_c, nc, best_c, pk_c + nc, pk_c + 2 * (size_t)nc, nullptr, st, flag_c)))
            return rc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st,
                   launch_fallback_seeds_list(fidx, flag_c, best_c, lib->quats, q, nc, seeds_c, st),
                   "fallback seeds");
        if ((rc = refine_chunk(ctx, lib, pat_c, nc, seeds_c, pc_c, q_c, pk_c, it_c, st, flag_c))) return rc;
        XCF_LAUNCH(XCF_STAGE_OTHER, st,
                   launch_fallback_scatter(fidx, flag_c, nc, q_c, pk_c, it_c, q, peak + p0, iters + p0, st),
                   "fallback results");
    }
    return XCF_OK;
}

// ------------------------------------------------------------- multi-map
namespace {

struct MapLayout {
    std::vector<size_t> spec, idx;   // offsets (complex values / patterns) of each map's slices
    size_t spec_total = 0, idx_total = 0;
};

MapLayout maps_layout(const xcf_map_desc *maps, int n) {
    MapLayout L;
    for (int m = 0; m < n; ++m) {
        const int N = maps[m].lib->N;
        L.spec.push_back(L.spec_total);
        L.idx.push_back(L.idx_total);
        L.spec_total += (size_t)maps[m].P * N * (N / 2 + 1);
        L.idx_total += (size_t)maps[m].P;
    }
    return L;
}

long long tune_key(int N, int T) { return ((long long)N << 32) | (unsigned)T; }

const xcf_ctx::Tuning *tuned(const xcf_ctx *ctx, int N, int T) {
    for (auto &kv : ctx->tune)
        if (kv.key == tune_key(N, T)) return &kv;
    return nullptr;
}

// sides served by the persistent queue: every side up to 160 x 160 (512-thread
// CTAs, one per SM, with shared memory for the largest body); 256 x 256 needs
// a four-CTA cluster, so those maps run the cluster kernel in the same stream
// (and graph)
bool queued_side(int N) { return N != 256 && N != 200; }

// the body and grouping a side runs before (or without) tuning: the body of
// its per-map kernel on whole CTAs
int default_body(int N) { return N == 128 ? kBodyRounds : N == 64 ? kBodyOct : N < 64 ? kBodySmem : kBodyReg; }
// whether G groups per CTA fit body b of side N (each group gets 1/G of the shared memory)
bool groups_fit(int N, int b, int G) {
    if (G != 1 && G != 2 && G != 4) return false;
    if (b == kBodyRounds) return G == 1;
    return maps_item_smem(N, b, kMapsThreads / G) <= ((maps_smem_bytes() / G) & ~(size_t)15);
}
int log2_groups(int G) { return G == 4 ? 2 : G == 2 ? 1 : 0; }

// one choice of the tuner (or of xcf_maps_set_tuning) for one map
struct Choice { int body, groups, pairs; };
Choice choice_of(const xcf_ctx *ctx, const xcf_library *lib) {
    const xcf_ctx::Tuning *t = tuned(ctx, lib->N, lib->T);
    if (t) return {t->body, t->groups, t->pairs};
    return {default_body(lib->N), 1, (lib->T + 1) / 2};
}

// the queue's items, ordered by phase (whole CTAs, two groups, four groups);
// within a phase the most expensive (largest detector) first, so that the
// tail of each phase is made of short items
struct ItemList {
    std::vector<WorkItem> v;
    int offs[4] = {0, 0, 0, 0};
};
// p_limit >= 0: at most that many patterns per map; only_map >= 0: that map
// alone, with the choice `force` if force.body >= 0
ItemList maps_items(xcf_ctx *ctx, const xcf_map_desc *maps, int n, int p_limit = -1, int only_map = -1,
                    Choice force = {-1, 1, 0}) {
    std::vector<int> order(n);
    for (int m = 0; m < n; ++m) order[m] = m;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return maps[a].lib->N > maps[b].lib->N; });
    std::vector<WorkItem> ph[3];
    for (int m : order) {
        if ((only_map >= 0 && m != only_map) || !queued_side(maps[m].lib->N)) continue;
        const int T = maps[m].lib->T, npairs = (T + 1) / 2;
        const Choice c = force.body >= 0 ? force : choice_of(ctx, maps[m].lib);
        const int pairs = c.pairs > 0 && c.pairs < npairs ? c.pairs : npairs;
        const int P = p_limit >= 0 && p_limit < maps[m].P ? p_limit : maps[m].P;
        std::vector<WorkItem> &out = ph[log2_groups(c.groups)];
        for (int p = 0; p < P; ++p)
            for (int pb = 0; pb < npairs; pb += pairs) out.push_back({m, p, pb, pb + pairs < npairs ? pb + pairs : npairs});
    }
    ItemList L;
    for (int k = 0; k < 3; ++k) {
        L.offs[k] = (int)L.v.size();
        L.v.insert(L.v.end(), ph[k].begin(), ph[k].end());
    }
    L.offs[3] = (int)L.v.size();
    return L;
}

struct MapsDev {
    MapDev *maps;
    WorkItem *items;
    int *counters;   // one per phase
    float2 *spec;
    int *degen;
    unsigned long long *keys;
    int grid;
};

// scratch for the batch (allocations happen here, never inside a capture)
int maps_scratch(xcf_ctx *ctx, const xcf_map_desc *maps, int n, const MapLayout &L, size_t n_items, MapsDev *d) {
    int rc;
    void *mp;
    const size_t table = ((sizeof(MapDev) * n + 255) & ~(size_t)255) + ((sizeof(WorkItem) * n_items + 255) & ~(size_t)255);
    if ((rc = scratch(ctx, S_MAPS, table + 256, &mp)) || (rc = scratch_t(ctx, S_SPEC_P, L.spec_total, &d->spec)) ||
        (rc = scratch_t(ctx, S_DEGEN, L.idx_total, &d->degen)) || (rc = scratch_t(ctx, S_KEYS, L.idx_total, &d->keys)))
        return rc;
    d->maps = static_cast<MapDev *>(mp);
    d->items = reinterpret_cast<WorkItem *>(static_cast<char *>(mp) + ((sizeof(MapDev) * n + 255) & ~(size_t)255));
    d->counters = reinterpret_cast<int *>(static_cast<char *>(mp) + table);
    if (ctx->opt.upsample >= 2) {   // the peak step's argmax scratch, sized before any capture
        int maxp = 1, *am;
        for (int m = 0; m < n; ++m) maxp = maps[m].P > maxp ? maps[m].P : maxp;
        if ((rc = scratch_t(ctx, S_ARGMAX, maxp, &am))) return rc;
    }
    d->grid = ctx->num_sms;
    return XCF_OK;
}

// force.body >= 0: that body for map only_map (the tuner's trials)
int maps_table_upload(xcf_ctx *ctx, const xcf_map_desc *maps, int n, const MapLayout &L, const MapsDev &d,
                      const ItemList &items, cudaStream_t st, int only_map = -1, Choice force = {-1, 1, 0}) {
    std::vector<MapDev> h(n);
    for (int m = 0; m < n; ++m) {
        const xcf_library *lib = maps[m].lib;
        const int body = force.body >= 0 && m == only_map ? force.body : choice_of(ctx, lib).body;
        h[m] = {lib->N, lib->T, body, lib->spectra, lib->spectra_pk, d.spec + L.spec[m], d.degen + L.idx[m],
                d.keys + L.idx[m]};
    }
    XCF_CHECK(cudaMemcpyAsync(d.maps, h.data(), sizeof(MapDev) * n, cudaMemcpyHostToDevice, st), "map table");
    if (!items.v.empty())
        XCF_CHECK(cudaMemcpyAsync(d.items, items.v.data(), sizeof(WorkItem) * items.v.size(), cudaMemcpyHostToDevice,
                                  st),
                  "work items");
    XCF_CHECK(cudaStreamSynchronize(st), "map table");
    return XCF_OK;
}

int maps_prep(xcf_ctx *ctx, const xcf_map_desc *maps, int n, const MapLayout &L, const MapsDev &d, cudaStream_t st) {
    for (int m = 0; m < n; ++m) {
        const xcf_library *lib = maps[m].lib;
        Crop c;
        crop_of(&lib->geom, 256, &c, lib->native);
        XCF_LAUNCH(XCF_STAGE_PREP, st,
                   run_prep(ctx, maps[m].patterns, maps[m].P, prep_args(&lib->geom, c, resolve(ctx->opt, c.n)),
                            d.spec + L.spec[m], nullptr, d.degen + L.idx[m], nullptr, st),
                   "prep");
    }
    return XCF_OK;
}

// the capturable part: search of all maps in one launch, then each map's peak
int maps_search_finish(xcf_ctx *ctx, const xcf_map_desc *maps, int n, const MapLayout &L, const MapsDev &d,
                       const ItemList &items, cudaStream_t st) {
    XCF_CHECK(cudaMemsetAsync(d.keys, 0, sizeof(unsigned long long) * L.idx_total, st), "clear keys");
    XCF_CHECK(cudaMemsetAsync(d.counters, 0, 3 * sizeof(int), st), "clear queue");
    if (!items.v.empty())
        XCF_LAUNCH(XCF_STAGE_SEARCH, st, launch_search_maps(d.maps, d.items, items.offs, d.counters, d.grid, st),
                   "multi-map search");
    for (int m = 0; m < n; ++m) {   // 256 x 256: the cluster kernel
        const xcf_library *lib = maps[m].lib;
        if (queued_side(lib->N)) continue;
        XCF_LAUNCH(XCF_STAGE_SEARCH, st,
                   run_search(ctx, lib->N, search_spectra(lib), lib->T, d.spec + L.spec[m], d.degen + L.idx[m],
                              maps[m].P, d.keys + L.idx[m], nullptr, ctx->num_sms, st),
                   "search");
    }
    for (int m = 0; m < n; ++m) {
        const xcf_library *lib = maps[m].lib;
        XCF_LAUNCH(XCF_STAGE_OTHER, st, launch_keys_to_best(d.keys + L.idx[m], maps[m].P, maps[m].best, st),
                   "keys_to_best");
        XCF_LAUNCH(XCF_STAGE_PEAK, st,
                   run_pair_peak(ctx, lib->N, lib->spectra, maps[m].best, d.spec + L.spec[m], d.degen + L.idx[m],
                                 nullptr, maps[m].P, maps[m].peak, maps[m].shift, st),
                   "pair_peak");
    }
    return XCF_OK;
}

// Time candidate (search body, groups per CTA, work granularity) choices on
// the first patterns of each untuned (side, library size) and keep the
// fastest (patterns already pre-processed).  Bodies: the line-transform
// decompositions the queue has for the side (128: three register rounds with
// shared-memory transposes, or warp lines of 4 x 32; 64: warp lines of
// 2 x 32, or radix-2 lines with the surface in shared memory).  Groups: 1, 2
// or 4 patterns side by side per CTA (each group on 512 / G threads and 1/G of
// the shared memory) where the body fits.  Granularity: template pairs per
// item.  Two stages: body and groups at a quarter of the library per item,
// then the granularity for the best of those.  The sample spans several waves
// of the persistent grid: finer items balance a short tail but break the
// library-order L2 reuse of a full-length sweep, and one wave alone
// overstates the first and hides the second.
constexpr int kTuneWaves = 8;
int maps_autotune(xcf_ctx *ctx, const xcf_map_desc *maps, int n, const MapLayout &L, const MapsDev &d,
                  cudaStream_t st) {
    cudaEvent_t e0, e1;
    XCF_CHECK(cudaEventCreate(&e0), "event");
    XCF_CHECK(cudaEventCreate(&e1), "event");
    int status = XCF_OK;
    const int sample = kTuneWaves * ctx->num_sms * 2;
    auto trial = [&](int m, Choice c, float *per) -> int {
        ItemList it = maps_items(ctx, maps, n, sample, m, c);
        int rc = maps_table_upload(ctx, maps, n, L, d, it, st, m, c);
        if (rc) return rc;
        cudaMemsetAsync(d.keys, 0, sizeof(unsigned long long) * L.idx_total, st);
        cudaMemsetAsync(d.counters, 0, 3 * sizeof(int), st);
        cudaEventRecord(e0, st);
        cudaError_t e = launch_search_maps(d.maps, d.items, it.offs, d.counters, d.grid, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const int pats = sample < maps[m].P ? sample : maps[m].P;
        *per = ms / (pats > 0 ? pats : 1);
        return XCF_OK;
    };
    for (int m = 0; m < n && status == XCF_OK; ++m) {
        const xcf_library *lib = maps[m].lib;
        const int N = lib->N, T = lib->T, npairs = (T + 1) / 2;
        if (!queued_side(N) || tuned(ctx, N, T)) continue;
        const int quarter = npairs / 4 > 8 ? npairs / 4 : (npairs < 8 ? npairs : 8);
        Choice best{default_body(N), 1, quarter};
        float best_t = 1e30f, per = 0.f;
        for (int body = 0; body < kNumBodies && status == XCF_OK; ++body) {
            if (!body_serves(N, body) || (body == kBodyRounds && !lib->spectra_pk)) continue;
            for (int G = 1; G <= 4 && status == XCF_OK; G *= 2) {
                if (!groups_fit(N, body, G)) continue;
                if ((status = trial(m, {body, G, quarter}, &per))) break;
                if (per < best_t) { best_t = per; best = {body, G, quarter}; }
            }
        }
        const int cands[2] = {npairs, npairs / 16 > 8 ? npairs / 16 : 8};
        for (int ci = 0; ci < 2 && status == XCF_OK; ++ci) {
            if (cands[ci] == quarter || cands[ci] > npairs) continue;
            Choice c = best;
            c.pairs = cands[ci];
            if ((status = trial(m, c, &per))) break;
            if (per < best_t) { best_t = per; best = c; }
        }
        if (status == XCF_OK) ctx->tune.push_back({tune_key(N, T), best.body, best.groups, best.pairs});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}

// launch shape of the queued items: persistent CTAs over the atomic queues
// (grid = SMs) or one CTA per 1, 2 or 4 items (grid = 0).  Timed on the first
// waves of the real item list and cached per batch configuration.
int maps_shape(xcf_ctx *ctx, const xcf_map_desc *maps, int n, const MapLayout &L, const MapsDev &d,
               const ItemList &items, const std::vector<char> &key, cudaStream_t st, int *grid) {
    for (auto &kv : ctx->shape_cache)
        if (kv.first == key) {
            *grid = kv.second;
            return XCF_OK;
        }
    *grid = d.grid;
    if (!items.v.empty()) {
        // a sample of each phase in proportion, kTuneWaves waves in all
        ItemList sample;
        const size_t want = (size_t)kTuneWaves * ctx->num_sms, total = items.v.size();
        for (int k = 0; k < 3; ++k) {
            sample.offs[k] = (int)sample.v.size();
            const size_t cnt = (size_t)(items.offs[k + 1] - items.offs[k]);
            const size_t take = total <= want ? cnt : (cnt * want + total - 1) / total;
            sample.v.insert(sample.v.end(), items.v.begin() + items.offs[k], items.v.begin() + items.offs[k] + take);
        }
        sample.offs[3] = (int)sample.v.size();
        int rc = maps_table_upload(ctx, maps, n, L, d, sample, st);
        if (rc) return rc;
        cudaEvent_t e0, e1;
        XCF_CHECK(cudaEventCreate(&e0), "event");
        XCF_CHECK(cudaEventCreate(&e1), "event");
        float best = 1e30f;
        const int shapes[2] = {d.grid, 0};
        for (int g : shapes) {
            cudaMemsetAsync(d.keys, 0, sizeof(unsigned long long) * L.idx_total, st);
            cudaMemsetAsync(d.counters, 0, 3 * sizeof(int), st);
            cudaEventRecord(e0, st);
            cudaError_t e = launch_search_maps(d.maps, d.items, sample.offs, d.counters, g, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(ctx, e, "launch-shape trial");
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                *grid = g;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    ctx->shape_cache.push_back({key, *grid});
    return XCF_OK;
}

}  // namespace

int xcf_maps_get_tuning(const xcf_ctx *ctx, int32_t N, int32_t T, int32_t *body, int32_t *groups,
                        int32_t *pairs) {
    if (!ctx || !body || !groups || !pairs) return XCF_ERR_ARG;
    const xcf_ctx::Tuning *t = tuned(ctx, N, T);
    if (!t) return XCF_ERR_ARG;
    *body = t->body;
    *groups = t->groups;
    *pairs = t->pairs;
    return XCF_OK;
}

int xcf_maps_set_tuning(xcf_ctx *ctx, int32_t N, int32_t T, int32_t body, int32_t groups, int32_t pairs) {
    if (!ctx) return XCF_ERR_ARG;
    if (!queued_side(N) || !body_serves(N, body) || !groups_fit(N, body, groups) || T <= 0 || pairs <= 0)
        return fail(ctx, XCF_ERR_ARG,
                    "xcf_maps_set_tuning: body not served for this side, groups not 1 / 2 / 4 or not fitting, or "
                    "T / pairs <= 0");
    const int npairs = (T + 1) / 2;
    if (pairs > npairs) pairs = npairs;
    for (auto it = ctx->tune.begin(); it != ctx->tune.end(); ++it)
        if (it->key == tune_key(N, T)) {
            ctx->tune.erase(it);
            break;
        }
    ctx->tune.push_back({tune_key(N, T), body, groups, pairs});
    // captured graphs and launch shapes were made with the previous items
    cudaSetDevice(ctx->device);
    drop_graph(ctx);
    ctx->shape_cache.clear();
    return XCF_OK;
}

int xcf_index_maps(xcf_ctx *ctx, const xcf_map_desc *maps, int32_t n_maps, int32_t flags, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (n_maps < 0 || (n_maps > 0 && !maps) || (flags & ~XCF_MAPS_GRAPH))
        return fail(ctx, XCF_ERR_ARG, "xcf_index_maps: bad argument");
    if (n_maps == 0) return XCF_OK;
    for (int m = 0; m < n_maps; ++m) {
        int rc = check_lib(ctx, maps[m].lib, true);
        if (rc) return rc;
        if (maps[m].P < 0 || (maps[m].P > 0 && (!maps[m].patterns || !maps[m].best || !maps[m].peak || !maps[m].shift)))
            return fail(ctx, XCF_ERR_ARG, "xcf_index_maps: bad map " + std::to_string(m));
    }
    cudaSetDevice(ctx->device);
    cudaStream_t caller = (cudaStream_t)stream;
    const MapLayout L = maps_layout(maps, n_maps);
    MapsDev d;
    int rc;

    // the key of this batch configuration (graph replay needs the same pointers and sizes)
    std::vector<char> key(reinterpret_cast<const char *>(maps), reinterpret_cast<const char *>(maps + n_maps));
    for (int m = 0; m < n_maps; ++m) {   // a library freed and another made at its address differs in id
        const uint64_t id = maps[m].lib->id;
        key.insert(key.end(), reinterpret_cast<const char *>(&id), reinterpret_cast<const char *>(&id) + sizeof id);
    }
    const bool graph = (flags & XCF_MAPS_GRAPH) != 0;
    if (graph && ctx->graph_exec && key == ctx->graph_key) {
        XCF_CHECK(cudaEventRecord(ctx->gev[0], caller), "event");
        XCF_CHECK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "event");
        // a replay is timed as one search-stage interval; its kernels are counted per stage
        XCF_LAUNCH(XCF_STAGE_SEARCH, ctx->gstream, cudaGraphLaunch(ctx->graph_exec, ctx->gstream), "graph launch");
        ctx->launches[XCF_STAGE_SEARCH] -= 1;
        for (int i = 0; i < XCF_NUM_STAGES; ++i) ctx->launches[i] += ctx->graph_launches[i];
        XCF_CHECK(cudaEventRecord(ctx->gev[1], ctx->gstream), "event");
        XCF_CHECK(cudaStreamWaitEvent(caller, ctx->gev[1], 0), "event");
        return XCF_OK;
    }

    // first call of this configuration: scratch, pre-processing, autotuning, work items
    ItemList items = maps_items(ctx, maps, n_maps);
    size_t max_items = items.v.size();
    for (int m = 0; m < n_maps; ++m)   // the largest trial list of the autotuner
        max_items = std::max(max_items, maps_items(ctx, maps, n_maps, 2 * kTuneWaves * ctx->num_sms, m,
                                                   {kBodyReg, 1, 8}).v.size());
    if ((rc = maps_scratch(ctx, maps, n_maps, L, max_items, &d))) return rc;
    if ((rc = maps_prep(ctx, maps, n_maps, L, d, caller))) return rc;
    if ((rc = maps_autotune(ctx, maps, n_maps, L, d, caller))) return rc;
    items = maps_items(ctx, maps, n_maps);   // the tuned granularity may need a larger table
    if (items.v.size() > max_items && (rc = maps_scratch(ctx, maps, n_maps, L, items.v.size(), &d))) return rc;
    if ((rc = maps_shape(ctx, maps, n_maps, L, d, items, key, caller, &d.grid))) return rc;
    if ((rc = maps_table_upload(ctx, maps, n_maps, L, d, items, caller))) return rc;

    if (!graph) return maps_search_finish(ctx, maps, n_maps, L, d, items, caller);

    // capture prep + search + peaks on the context's own stream, then replay
    if (!ctx->gstream) XCF_CHECK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking), "stream");
    for (auto &e : ctx->gev)
        if (!e) XCF_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    drop_graph(ctx);
    XCF_CHECK(cudaStreamSynchronize(caller), "sync");
    const bool timing = ctx->timing;
    ctx->timing = false;   // no event pairs inside the capture
    int64_t before[XCF_NUM_STAGES];
    for (int i = 0; i < XCF_NUM_STAGES; ++i) before[i] = ctx->launches[i];
    XCF_CHECK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal), "begin capture");
    rc = maps_prep(ctx, maps, n_maps, L, d, ctx->gstream);
    if (rc == XCF_OK) rc = maps_search_finish(ctx, maps, n_maps, L, d, items, ctx->gstream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->gstream, &g);
    ctx->timing = timing;
    for (int i = 0; i < XCF_NUM_STAGES; ++i) ctx->graph_launches[i] = ctx->launches[i] - before[i];
    if (rc != XCF_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ec != cudaSuccess) return cuda_fail(ctx, ec, "end capture");
    XCF_CHECK(cudaGraphInstantiate(&ctx->graph_exec, g, 0), "graph instantiate");
    ctx->graph = g;
    ctx->graph_key = key;
    XCF_CHECK(cudaGraphLaunch(ctx->graph_exec, ctx->gstream), "graph launch");
    XCF_CHECK(cudaEventRecord(ctx->gev[1], ctx->gstream), "event");
    XCF_CHECK(cudaStreamWaitEvent(caller, ctx->gev[1], 0), "event");
    return XCF_OK;
}

}  // extern "C"
