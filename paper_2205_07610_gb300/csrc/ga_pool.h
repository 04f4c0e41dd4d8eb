// ga_pool.h -- the library's stream-ordered device memory pool (one per
// device, created on first use, freed memory kept mapped between calls).
#pragma once

#include <cuda_runtime.h>

namespace ga {

cudaMemPool_t pool_for_current_device();
cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t s);

}  // namespace ga
