// Device and pinned host memory of the library's contexts.
//
// Device buffers come from one stream-ordered memory pool per device, owned
// by the library, whose release threshold keeps freed memory cached: a field
// after the first reuses the memory of the contexts before it, without a
// cudaMalloc / cudaFree (which synchronises the device) per buffer, and
// allocation and release are ordered on the context's stream.
// mpr_release_cached_memory hands the cached part back to the device.
//
// The few bytes of pinned host memory a context reads its counters into come
// from one pinned slab shared by all contexts, in fixed slots.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "mpr_memory.h"

namespace mpr {
namespace {

std::mutex g_mu;
std::vector<cudaMemPool_t> g_pools;      // by device ordinal (nullptr: not created)

constexpr size_t kSlots = 4096;
uint8_t* g_slab = nullptr;                // kSlots * kPinnedSlot bytes of pinned memory
std::vector<uint32_t> g_free_slots;

cudaMemPool_t pool_for(int device) {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_pools.size() <= device) g_pools.resize(device + 1, nullptr);
    if (g_pools[device]) return g_pools[device];
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[device] = p;
    return p;
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, int device, cudaStream_t s) {
    *p = nullptr;
    cudaMemPool_t pool = pool_for(device);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void pool_trim() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (cudaMemPool_t p : g_pools)
        if (p) cudaMemPoolTrimTo(p, 0);
}

void* pinned_slot() {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_slab) {
            void* q = nullptr;
            if (cudaMallocHost(&q, kSlots * kPinnedSlot) == cudaSuccess) {
                g_slab = static_cast<uint8_t*>(q);
                g_free_slots.reserve(kSlots);
                for (size_t i = kSlots; i-- > 0;) g_free_slots.push_back((uint32_t)i);
            } else {
                cudaGetLastError();
            }
        }
        if (g_slab && !g_free_slots.empty()) {
            const uint32_t i = g_free_slots.back();
            g_free_slots.pop_back();
            return g_slab + (size_t)i * kPinnedSlot;
        }
    }
    void* q = nullptr;                     // slab exhausted: a slot of its own
    if (cudaMallocHost(&q, kPinnedSlot) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}

void pinned_release(void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const uint8_t* b = static_cast<const uint8_t*>(p);
        if (g_slab && b >= g_slab && b < g_slab + kSlots * kPinnedSlot) {
            g_free_slots.push_back((uint32_t)((b - g_slab) / kPinnedSlot));
            return;
        }
    }
    cudaFreeHost(p);
}

}  // namespace mpr
