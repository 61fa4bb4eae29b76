// Definitions of the opaque handles of the ebsdxcf C ABI, shared by the host
// translation units of the library (not part of the public interface).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ebsdxcf.h"

namespace xcf_internal {

constexpr double kPi = 3.14159265358979323846;

// slots of the per-context grow-only scratch arena
enum Slot {
    S_SPEC_P = 0,   // pattern half spectra
    S_SPEC_T,       // per-pattern template half spectra (refinement)
    S_SPATIAL_P,    // filtered pattern images
    S_SPATIAL_T,    // filtered template images
    S_IMG,          // projected template images
    S_LP_P,         // log-polar patterns
    S_LP_T,         // log-polar templates
    S_KEYS,
    S_DEGEN,
    S_ACTIVE,
    S_SHIFT,
    S_Q1,
    S_SEEDS,
    S_BEST,
    S_PEAK,
    S_IO_PAT,       // host pipeline: device copy of a chunk of patterns
    S_IO_PCS,
    S_IO_OUT,
    S_BF16_P,       // screen: pattern images in BF16
    S_SCORE,        // screen: zero-shift scores of a chunk
    S_ERR,          // device status word of kernels with bounded waits
    S_MAPS,         // multi-map search: map table, work items, queue counter
    S_PROP,         // learned proposals [P, k, 4]
    S_QH,           // one proposal per pattern [P, 4]
    S_BESTPEAK,     // best proposal peak [P]
    S_MASK,         // search mask of the fallback pass
    S_FBCOUNT,      // fallback patterns and fallback pattern pairs (two device ints)
    S_FB_IDX,       // fallback pass: the batch's pattern indices (by pairs)
    S_FB_FLAG,      // fallback pass: which of them are flagged
    S_FB_PAT,       // fallback pass: their images
    S_FB_PC,        // fallback pass: their pattern centres
    S_FB_BEST,      // fallback pass: their best templates
    S_FB_PEAK,      // fallback pass: refined peak, best peak, shift (x, y) per pattern
    S_FB_Q,         // fallback pass: refined orientations, then seeds
    S_FB_IT,        // fallback pass: iteration counts
    S_CAND,         // screen candidates of a chunk [P, k]
    S_CANDSC,       // their screen scores
    S_ARGMAX,       // integer peak positions for the up-sampled peak
    S_BG_TMP,       // NDP background correction: row-blurred crops
    S_BG_OUT,       // NDP background correction: corrected crops
    S_SO3_RING,     // SO(3) generator: ring starts and azimuth counts
    S_SO3_QALL,     // SO(3) generator: every grid point [G][4]
    S_SO3_QFZ,      // SO(3) generator: the points in the fundamental zone
    S_SO3_FLAG,     // SO(3) generator: keep flags
    S_SO3_CNT,      // SO(3) generator: compaction block counts + total
    S_NN_KEYS,      // nearest neighbour: packed best keys
    S_NN_ANG,       // nearest neighbour: angles (generator's duplicate pass)
    S_NN_IDX,       // nearest neighbour: indices (generator's duplicate pass)
    S_NET_BF16,     // proposal network, BF16 inference: the convolutions' BF16 weights [Co][Kp]
    S_PROBE,        // FMA rate probe: its sink word
    S_COUNT
};

}  // namespace xcf_internal

struct xcf_ctx {
    int device = 0;
    int num_sms = 0;
    xcf_options opt{};
    std::string err;
    void *buf[xcf_internal::S_COUNT] = {};
    size_t cap[xcf_internal::S_COUNT] = {};
    size_t scratch_limit = 0;   // 0: no cap on the sum of cap[]
    // profiling
    bool timing = false;
    int64_t launches[XCF_NUM_STAGES] = {};
    double ms[XCF_NUM_STAGES] = {};
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    // multi-map search: autotuned search body and template pairs per work item,
    // keyed by (N, T), and the chosen launch shape per batch configuration
    struct Tuning { long long key; int body; int groups; int pairs; };
    std::vector<Tuning> tune;
    std::vector<std::pair<std::vector<char>, int>> shape_cache;
    // multi-map search: captured graph of the last batch configuration
    std::vector<char> graph_key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches[XCF_NUM_STAGES] = {};   // kernels of one replay, per stage
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
};

inline uint64_t next_library_id() {
    static std::atomic<uint64_t> n{0};
    return ++n;
}

struct xcf_library {
    uint64_t id = next_library_id();   // unique per library made in this process
    int device = 0;
    int T = 0, N = 0, M = 0;
    bool native = false;               // crop rule of the context that built it (native 96 / 160 sides)
    xcf_geometry geom{};
    int ox = 0, oy = 0;
    double pc[3] = {0, 0, 0};
    float2 *spectra = nullptr;
    float2 *spectra_pk = nullptr;   // N = 128 and 256: the search kernel's layout (always made with spectra)
    void *bf16 = nullptr;           // screen: unit-norm filtered images [T][N*N] in BF16
    float *ndp32 = nullptr;         // NDP: contrast-normalised images / N [T][N*N] in FP32 ...
    void *ndp16 = nullptr;          // ... and in BF16 (inside the same allocation)
    double *quats = nullptr;
    float *master = nullptr;
};

// sides whose search kernel reads the templates in a layout of its own, and
// that layout's float2 per template
size_t c256_search_layout_f2();   // k_c256.cu
inline bool has_search_layout(int n) { return n == 128 || n == 256; }
inline size_t search_layout_f2(int n) { return n == 256 ? c256_search_layout_f2() : (size_t)n * (n / 2 + 1); }

// spectra as the all-pairs search kernel of the library's size reads them
inline const float2 *search_spectra(const xcf_library *lib) {
    return lib->spectra_pk ? lib->spectra_pk : lib->spectra;
}

// the proposal network: parameters, Adam state and grow-only work buffers
struct xcf_net {
    int device = 0;
    int k = 0;
    int bf16 = 0;                   // inference forward: 0 FP32, 1 BF16 tensor-core convolutions
    long n = 0;                     // parameter count
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // [n] each, one allocation
    int t = 0;                      // Adam steps taken
    float *act = nullptr;           // activations of the last forward
    size_t act_cap = 0;
    float *gbuf = nullptr;          // gradient work buffers
    size_t gbuf_cap = 0;
};
