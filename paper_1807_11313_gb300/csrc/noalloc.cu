// Library search that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely
// owned by another allocator (for example a framework's caching allocator
// that has reserved the GPU), and latency-critical loops that cannot accept
// the device-wide synchronisation cudaMalloc / cudaFree bring.  For them,
// xcf_index_noalloc runs exactly the kernels of xcf_index, but keeps its
// scratch (pattern spectra, degeneracy flags, best-template keys) in the
// fixed array below, compiled into the library.  Every GPU that loads the
// library holds this array until the process exits.  CUDA loads a library's
// modules lazily by default, so the array (with this file's small module) is
// committed on a device by the first call there, not at library load: that
// first call must come before another allocator reserves the GPU, and before
// any stream capture.
#include <cuda.h>

#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)XCF_NOALLOC_SCRATCH_BYTES;

// the scratch of every xcf_index_noalloc call on a device (shared by calls)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// device address of g_noalloc_scratch per device, and the CUDA context it was
// looked up in (a device reset or a new primary context loads the module
// again, possibly elsewhere: the address is then looked up anew)
void *g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// unique id of the current CUDA context (0 if it cannot be had)
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // under g_mutex
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
        cudaGetLastError();
        looked_up = true;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of scratch for P patterns of side n: spectra | flags | keys
size_t scratch_bytes(int n, long P) {
    const size_t H = (size_t)n * (n / 2 + 1);
    return round_up(sizeof(float2) * H * P) + round_up(sizeof(int) * P) +
           round_up(sizeof(unsigned long long) * P);
}

// One-time set-up per device and CUDA context (the device is current): the
// host-side name of the array is only a stand-in, so look up its device
// address (which loads this file's module on the first call).
int device_scratch(xcf_ctx *ctx, void **out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices) {
        ctx->err = "xcf_index_noalloc: device ordinal out of range";
        return XCF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long id = current_context_id();
    if (!g_addr[ctx->device] || id == 0 || id != g_ctx_id[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            ctx->err = std::string("xcf_index_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return XCF_ERR_CUDA;
        }
        g_addr[ctx->device] = p;
        g_ctx_id[ctx->device] = id;
    }
    *out = g_addr[ctx->device];
    return XCF_OK;
}

int cuda_error(xcf_ctx *ctx, cudaError_t e, const char *where) {
    ctx->err = std::string("xcf_index_noalloc: ") + where + ": " + cudaGetErrorString(e);
    return XCF_ERR_CUDA;
}

// one launch of `stage`: counted, and timed with an event pair when the
// context's timing is on (as every other entry point's launches)
template <class F>
int launch(xcf_ctx *ctx, int stage, cudaStream_t st, F &&fn, const char *where) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (ctx->timing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
    const cudaError_t e = fn();
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_error(ctx, e, where);
    }
    ctx->launches[stage] += 1;
    if (a && cudaEventCreate(&b) == cudaSuccess) {
        cudaEventRecord(b, st);
        ctx->recs.push_back({stage, a, b});
    } else if (a) {
        cudaEventDestroy(a);
    }
    return XCF_OK;
}

}  // namespace

extern "C" int xcf_noalloc_max_patterns(int32_t n) {
    // every side the kernels take: 2^k in [16, 256] and the native 96 and 160
    if (!(n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 256)) return 0;
    long lo = 0, hi = 1L << 24;
    while (lo < hi) {       // largest P whose scratch fits
        long mid = (lo + hi + 1) / 2;
        if (scratch_bytes(n, mid) <= kScratchBytes) lo = mid; else hi = mid - 1;
    }
    return (int)lo;
}

extern "C" int xcf_index_noalloc(xcf_ctx *ctx, const xcf_library *lib, const float *patterns, int32_t P,
                                 int32_t *best, float *peak, float *shift, void *stream) {
    if (!ctx) return XCF_ERR_ARG;
    if (!lib) { ctx->err = "xcf_index_noalloc: library is NULL"; return XCF_ERR_ARG; }
    if (lib->device != ctx->device) { ctx->err = "xcf_index_noalloc: library on another device"; return XCF_ERR_ARG; }
    if (!lib->spectra) { ctx->err = "xcf_index_noalloc: library built with XCF_LIB_NO_SPECTRA"; return XCF_ERR_ARG; }
    if (P == 0) return XCF_OK;
    if (!patterns || !best || !peak || !shift || P < 0) {
        ctx->err = "xcf_index_noalloc: bad argument";
        return XCF_ERR_ARG;
    }
    const int n = lib->N;
    if (ctx->opt.upsample >= 2) {
        ctx->err = "xcf_index_noalloc: the up-sampled peak needs scratch; use xcf_index";
        return XCF_ERR_UNIMPLEMENTED;
    }
    const int pmax = xcf_noalloc_max_patterns(n);
    if (P > pmax) {
        ctx->err = "xcf_index_noalloc: " + std::to_string(P) + " patterns exceed the fixed scratch (" +
                   std::to_string(pmax) + " patterns of " + std::to_string(n) + " x " + std::to_string(n) +
                   " fit in " + std::to_string(kScratchBytes) + " bytes); split the call or use xcf_index";
        return XCF_ERR_SIZE;
    }
    cudaSetDevice(ctx->device);
    void *base = nullptr;
    int rc = device_scratch(ctx, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    // carve the fixed array: spectra | flags | keys
    const size_t H = (size_t)n * (n / 2 + 1);
    unsigned char *b = static_cast<unsigned char *>(base);
    float2 *sp = reinterpret_cast<float2 *>(b);
    int *degen = reinterpret_cast<int *>(b + round_up(sizeof(float2) * H * P));
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(
        b + round_up(sizeof(float2) * H * P) + round_up(sizeof(int) * P));

    // the same pre-processing arguments as xcf_index
    const xcf_geometry *g = &lib->geom;
    const xcf_options &o = ctx->opt;
    const double shp = o.sigma_hp > 0 ? o.sigma_hp : 2.0;
    const double slp = o.sigma_lp > 0 ? o.sigma_lp : n / 4.0;
    PrepArgs a;
    a.N = n;
    a.W = g->width;
    a.H = g->height;
    a.ox = lib->ox;
    a.oy = lib->oy;
    a.window = o.window;
    a.inv2shp = (float)(1.0 / (2.0 * shp * shp));
    a.inv2slp = (float)(1.0 / (2.0 * slp * slp));

    // N = 256 runs on four-CTA clusters, which need no scratch beyond the spectra
    const bool c256 = n == 256;
    if ((rc = launch(ctx, XCF_STAGE_PREP, st, [&] {
             return c256 ? launch_prep_c256(patterns, P, a, sp, nullptr, degen, nullptr, st)
                         : launch_prep(patterns, P, a, sp, nullptr, degen, nullptr, st);
         }, "prep")))
        return rc;
    // the array keeps the previous call's contents: the keys must start at 0
    const cudaError_t e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * P, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "clear keys");
    if ((rc = launch(ctx, XCF_STAGE_SEARCH, st, [&] {
             return c256 ? launch_search_c256(search_spectra(lib), lib->T, sp, degen, P, keys, nullptr, nullptr, 0, st)
                         : launch_search(n, search_spectra(lib), lib->T, sp, degen, P, keys, nullptr, ctx->num_sms,
                                         st);
         }, "search")))
        return rc;
    if ((rc = launch(ctx, XCF_STAGE_OTHER, st, [&] { return launch_keys_to_best(keys, P, best, st); },
                     "keys_to_best")))
        return rc;
    return launch(ctx, XCF_STAGE_PEAK, st, [&] {
        return c256 ? launch_pair_peak_c256(lib->spectra, best, sp, degen, nullptr, P, peak, shift, st)
                    : launch_pair_peak(n, lib->spectra, best, sp, degen, nullptr, P, peak, shift, st);
    }, "pair_peak");
}
