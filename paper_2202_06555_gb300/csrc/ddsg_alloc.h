// ddsg_alloc.h -- the one device-allocation routine of libddsg. Every entry point
// allocates through it so that a test switch (ddsg_inject_alloc_failure) can make
// allocations fail the way an exhausted device does, without touching the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace ddsg {
// cudaMalloc, or cudaErrorMemoryAllocation with *ptr = nullptr when the switch
// says this allocation fails.
cudaError_t dev_alloc(void **ptr, size_t bytes);
template <typename T>
inline cudaError_t dev_alloc(T **ptr, size_t bytes) {
    return dev_alloc(reinterpret_cast<void **>(ptr), bytes);
}
}  // namespace ddsg
