// Memory of the library's contexts (mpr_memory.cu): stream-ordered device
// allocations from a per-device pool that caches freed memory, and fixed
// pinned host slots for counter readbacks.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace mpr {

constexpr size_t kPinnedSlot = 256;   // bytes of one pinned host slot

// Allocates `bytes` on `device`, ordered on stream s (usable by work queued
// on s after this call).
cudaError_t pool_alloc(void** p, size_t bytes, int device, cudaStream_t s);
// Returns p to the pool once the work queued on s before this call is done.
void pool_free(void* p, cudaStream_t s);
// Releases the pools' cached memory to the device.
void pool_trim();

// A pinned host slot of kPinnedSlot bytes (contents undefined), or nullptr.
void* pinned_slot();
void pinned_release(void* p);

}  // namespace mpr
