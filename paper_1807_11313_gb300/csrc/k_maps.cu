// Several maps with different detectors searched in one persistent launch.
//
// Paper: the search of Fig. 1 B-C applied to many maps at once (the maps of
// the Demonstrations section have different pattern centres and sizes; the
// crop to 2^n of the FFT section maps 96 -> 64, 160 / 200 -> 128 px).
//
// One CTA per SM loops over a queue of work items (map, pattern, range of
// template pairs), taken with an atomic counter, and runs the search body of
// that map's detector side: the tuned 128 x 128 kernel's body, the generic
// shared-memory body (16..64) or the global-work-array body (256).  A CTA
// never waits for another: the queue only hands out indices.
#include "big.cuh"
#include "common.cuh"
#include "generic.cuh"
#include "kernels.cuh"
#include "search128.cuh"

namespace {

constexpr int kMapThreads = 256;
static_assert(s128::NT == kMapThreads && gen::kThreads == kMapThreads && bigk::kThreads == kMapThreads,
              "all search bodies run on 256 threads");
static_assert(gen::smem_bytes<64>() <= s128::SMEM_BYTES && bigk::smem_big(256) <= s128::SMEM_BYTES,
              "every body fits the launch's dynamic shared memory");

__global__ void __launch_bounds__(kMapThreads, 1)
k_search_maps(const MapDev *__restrict__ maps, const WorkItem *__restrict__ items, int n_items, int *counter,
              float2 *__restrict__ work) {
    extern __shared__ float4 smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ int s_item;
    __shared__ float redf[33];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();   // every thread has the index before thread 0 takes the next
        if (it >= n_items) break;
        const WorkItem w = items[it];
        const MapDev m = maps[w.map];
        if (m.degen[w.p]) continue;
        switch (m.N) {
            case 128: s128::search_body(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr); break;
            case 64: gen::search_body<64>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0); break;
            case 32: gen::search_body<32>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0); break;
            case 16: gen::search_body<16>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr, nullptr, 0); break;
            case 256: {
                float2 *tw = sm + (size_t)256 * bigk::kColTile;
                bigk::make_tw<256>(tw, +1);
                __syncthreads();
                bigk::search_body<256>(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr,
                                       work + (size_t)blockIdx.x * 256 * 256, sm, tw, redf, nullptr, 0);
                break;
            }
            default: break;
        }
        __syncthreads();   // the item's shared memory is free for the next one
    }
}

}  // namespace

size_t maps_smem_bytes() { return s128::SMEM_BYTES; }

cudaError_t launch_search_maps(const MapDev *maps, const WorkItem *items, int n_items, int *counter, float2 *work,
                               int grid, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_search_maps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)maps_smem_bytes());
    if (e != cudaSuccess) return e;
    k_search_maps<<<grid, kMapThreads, maps_smem_bytes(), st>>>(maps, items, n_items, counter, work);
    return cudaGetLastError();
}
