// Several maps searched in one persistent launch.
//
// Paper: the search of Fig. 1 B-C applied to many maps at once (the maps of
// the Demonstrations section have different pattern centres and sizes; the
// crop of the FFT section maps 96 -> 64 and 160 / 200 -> 128 px, or keeps 96
// and 160 with the native crop rule).
//
// One CTA per SM (512 threads, shared memory sized for the largest side)
// loops over a queue of work items (map, pattern, range of template pairs)
// of every map of the batch up to 160 x 160, taken with an atomic counter;
// each item runs the search body its map's side and tuning name:
//   kBodyRounds  N = 128, three register rounds with two shared-memory
//                transposes (16 x 8 columns, 4 x 32 rows);
//   kBodyReg     N = R x 32 (64, 96, 128, 160), rows and columns as warp-line
//                transforms in registers (R points per lane, 32-point lane
//                stages by shuffles);
//   kBodySmem    N = 2^k <= 64, the surface in shared memory with radix-2
//                line transforms;
//   kBodyOct     N = 64, eight-lane groups: 8-point transforms in registers
//                joined by shared-memory transposes (oct64.cuh).
// The maps may have different libraries, pattern centres and detectors.  A
// CTA never waits for another: the queue only hands out indices.  The
// alternative launch shape (one CTA per item, grid = items) is one of the
// autotuner's candidates.  (256 x 256 maps need four-CTA clusters and run
// the cluster kernel: see queued_side in api.cu.)
#include "common.cuh"
#include "kernels.cuh"
#include "generic.cuh"
#include "search128.cuh"
#include "oct64.cuh"

namespace {

constexpr int kMapThreads = s128::NT;
static_assert(kMapThreads == kMapsThreads, "the queue CTA runs the three-round 128 body on all its threads");

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kMapsSmem = cmax(cmax(s128::SMEM_BYTES, gen::smem_bytes<160>()),
                                  cmax(gen::smem_bytes<128>(), gen::smem_bytes<96>()));
static_assert(o64::smem_bytes(kMapThreads) <= kMapsSmem, "the 8 x 8 body fits a whole queue CTA");

__device__ __forceinline__ void run_item(const MapDev &m, const WorkItem &w, const gen::Grp &g) {
    switch (m.N) {
        case 16: gen::search_body_smem<16>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g); break;
        case 32: gen::search_body_smem<32>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g); break;
        case 64:
            if (m.body == kBodySmem)
                gen::search_body_smem<64>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g);
            else if (m.body == kBodyOct)
                o64::search_body(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g);
            else
                gen::search_body_reg<64>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g);
            break;
        case 96: gen::search_body_reg<96>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g); break;
        case 128:
            if (m.body == kBodyRounds)   // whole CTAs only (phase 0)
                s128::search_body(m.Stp, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr);
            else
                gen::search_body_reg<128>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g);
            break;
        case 160: gen::search_body_reg<160>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0, g); break;
        default: break;   // not a queued side (the host never enqueues one)
    }
}

// group gid of 2^ph equal groups of the CTA, with its slice of the shared memory
__device__ __forceinline__ gen::Grp phase_group(int ph, int &gid) {
    extern __shared__ float4 smem_raw[];
    const int G = 1 << ph, gn = kMapThreads / G;
    gid = (int)threadIdx.x / gn;
    const size_t region = (kMapsSmem / G) & ~(size_t)15;
    return gen::Grp{(int)threadIdx.x - gid * gn, gn, G == 1 ? 0 : 1 + gid,
                    reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem_raw) + gid * region)};
}

// one CTA per 1, 2 or 4 items (the hardware block scheduler balancing)
__global__ void __launch_bounds__(kMapThreads, 1)
k_search_items(const MapDev *__restrict__ maps, const WorkItem *__restrict__ items, int4 offs, int b1, int b2) {
    // blocks [0, b1): phase 0; [b1, b2): phase 1; [b2, ...): phase 2
    const int b = blockIdx.x;
    const int ph = b < b1 ? 0 : b < b2 ? 1 : 2;
    const int lo = ph == 0 ? offs.x : ph == 1 ? offs.y : offs.z;
    const int hi = ph == 0 ? offs.y : ph == 1 ? offs.z : offs.w;
    const int first = ph == 0 ? b : ph == 1 ? b - b1 : b - b2;
    int gid;
    const gen::Grp g = phase_group(ph, gid);
    const int it = lo + (first << ph) + gid;
    if (it >= hi) return;   // whole groups leave together
    const WorkItem w = items[it];
    const MapDev m = maps[w.map];
    if (m.degen[w.p]) return;
    run_item(m, w, g);
}

__global__ void __launch_bounds__(kMapThreads, 1)
k_search_maps(const MapDev *__restrict__ maps, const WorkItem *__restrict__ items, int4 offs, int *counters) {
    __shared__ int s_item[4];
    const int bounds[4] = {offs.x, offs.y, offs.z, offs.w};
    for (int ph = 0; ph < 3; ++ph) {
        const int lo = bounds[ph], hi = bounds[ph + 1];
        if (lo >= hi) continue;   // uniform over the CTA
        int gid;
        const gen::Grp g = phase_group(ph, gid);
        for (;;) {
            if (g.t == 0) s_item[gid] = lo + atomicAdd(counters + ph, 1);
            g.sync();
            const int it = s_item[gid];
            g.sync();   // every thread of the group has the index before its leader takes the next
            if (it >= hi) break;
            const WorkItem w = items[it];
            const MapDev m = maps[w.map];
            if (!m.degen[w.p]) run_item(m, w, g);
            g.sync();   // the item's shared memory is free for the group's next one
        }
        __syncthreads();   // every group is out of this phase before the shared memory is cut anew
    }
}

}  // namespace

size_t maps_smem_bytes() { return kMapsSmem; }

cudaError_t launch_search_maps(const MapDev *maps, const WorkItem *items, const int offs[4], int *counters,
                               int grid, cudaStream_t st) {
    if (offs[3] <= offs[0]) return cudaSuccess;
    const int4 o = make_int4(offs[0], offs[1], offs[2], offs[3]);
    if (grid <= 0) {   // one CTA per 1, 2 or 4 items
        const int b1 = offs[1] - offs[0], b2 = b1 + (offs[2] - offs[1] + 1) / 2;
        const int blocks = b2 + (offs[3] - offs[2] + 3) / 4;
        cudaError_t e = cudaFuncSetAttribute(k_search_items, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)maps_smem_bytes());
        if (e != cudaSuccess) return e;
        k_search_items<<<blocks, kMapThreads, maps_smem_bytes(), st>>>(maps, items, o, b1, b2);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_search_maps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)maps_smem_bytes());
    if (e != cudaSuccess) return e;
    k_search_maps<<<grid, kMapThreads, maps_smem_bytes(), st>>>(maps, items, o, counters);
    return cudaGetLastError();
}
