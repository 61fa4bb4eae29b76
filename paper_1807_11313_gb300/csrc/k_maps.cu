// Several maps searched in one persistent launch.
//
// Paper: the search of Fig. 1 B-C applied to many maps at once (the maps of
// the Demonstrations section have different pattern centres and sizes; the
// crop to 2^n of the FFT section maps 160 / 200 -> 128 px).
//
// One CTA per SM loops over a queue of work items (map, pattern, range of
// template pairs) of every 128 x 128 map of the batch, taken with an atomic
// counter, and runs the tuned 128 x 128 body on each; the maps may have
// different libraries, pattern centres and detectors.  A CTA never waits for
// another: the queue only hands out indices.  The alternative launch shape
// (one CTA per item, grid = items) is one of the autotuner's candidates.  (Maps of other sides run their
// own kernels in the same stream: see queued_side in api.cu.)
#include "common.cuh"
#include "kernels.cuh"
#include "search128.cuh"

namespace {

constexpr int kMapThreads = s128::NT;

// one item per CTA (grid = items), the hardware block scheduler balancing
__global__ void __launch_bounds__(kMapThreads, 1)
k_search_items(const MapDev *__restrict__ maps, const WorkItem *__restrict__ items) {
    const WorkItem w = items[blockIdx.x];
    const MapDev m = maps[w.map];
    if (m.degen[w.p] || m.N != 128) return;
    s128::search_body(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr);
}

__global__ void __launch_bounds__(kMapThreads, 1)
k_search_maps(const MapDev *__restrict__ maps, const WorkItem *__restrict__ items, int n_items, int *counter,
              float2 *__restrict__ work) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();   // every thread has the index before thread 0 takes the next
        if (it >= n_items) break;
        const WorkItem w = items[it];
        const MapDev m = maps[w.map];
        if (m.degen[w.p] || m.N != 128) continue;
        s128::search_body(m.St, m.T, m.Sp, w.p, w.pb, w.pe, m.keys, nullptr);
        __syncthreads();   // the item's shared memory is free for the next one
    }
}

}  // namespace

size_t maps_smem_bytes() { return s128::SMEM_BYTES; }

cudaError_t launch_search_maps(const MapDev *maps, const WorkItem *items, int n_items, int *counter, float2 *work,
                               int grid, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (grid <= 0) {   // one CTA per item
        cudaError_t e = cudaFuncSetAttribute(k_search_items, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)maps_smem_bytes());
        if (e != cudaSuccess) return e;
        k_search_items<<<n_items, kMapThreads, maps_smem_bytes(), st>>>(maps, items);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_search_maps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)maps_smem_bytes());
    if (e != cudaSuccess) return e;
    k_search_maps<<<grid, kMapThreads, maps_smem_bytes(), st>>>(maps, items, n_items, counter, work);
    return cudaGetLastError();
}
