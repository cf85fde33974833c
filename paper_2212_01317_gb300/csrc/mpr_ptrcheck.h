// Which pointers the allocation-free entry point accepts, as a plain function
// of the pointer's attributes so that host code without a GPU can test it.
//
// A caller's buffer is usable by kernels launched on the current device when
// it is device memory of that same device, or managed memory. Device memory
// of another device would be read from the wrong GPU (without peer access, an
// illegal address), so it is rejected like a host pointer.
#pragma once
#include <cuda_runtime_api.h>

namespace mpr {

inline bool noalloc_pointer_ok(cudaMemoryType type, int owner_device, int current_device) {
    if (type == cudaMemoryTypeManaged) return true;
    return type == cudaMemoryTypeDevice && owner_device == current_device;
}

}  // namespace mpr
