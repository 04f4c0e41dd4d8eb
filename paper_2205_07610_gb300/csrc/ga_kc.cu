// Banded (band-doubling) kernel instantiations: int32 and packed int16x2.
#include "ga_bandcz.cuh"
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

cudaError_t launch_kz(const KCParams &p, int grid, cudaStream_t s) {
  kz_kernel<kKcK><<<grid, kKcThreads, 0, s>>>(p);
  return cudaGetLastError();
}

int blocks_per_sm_kz() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kz_kernel<kKcK>, kKcThreads, 0);
  return n;
}

}  // namespace ga
