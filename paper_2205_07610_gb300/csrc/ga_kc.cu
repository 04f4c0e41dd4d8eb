// Banded (band-doubling) kernel instantiations: int32 and packed int16x2.
#include "ga_bandpk.cuh"
#include "ga_banded.cuh"
#include "ga_launch.h"

namespace ga {

cudaError_t launch_kc(const KCParams &p, int grid, cudaStream_t s) {
  kc_kernel<kKcK><<<grid, kKcThreads, 0, s>>>(p);
  return cudaGetLastError();
}

int blocks_per_sm_kc() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kc_kernel<kKcK>, kKcThreads, 0);
  return n;
}

cudaError_t launch_kd(const KCParams &p, int grid, cudaStream_t s, bool narrow) {
  if (narrow) kd_kernel<kKcK, kKdGNarrow><<<grid, kKcThreads, 0, s>>>(p);
  else kd_kernel<kKcK, kKdGWide><<<grid, kKcThreads, 0, s>>>(p);
  return cudaGetLastError();
}

int blocks_per_sm_kd(bool narrow) {
  int n = 0;
  if (narrow) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kd_kernel<kKcK, kKdGNarrow>, kKcThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kd_kernel<kKcK, kKdGWide>, kKcThreads, 0);
  return n;
}

}  // namespace ga
