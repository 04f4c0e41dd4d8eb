// Packed int16x2 long-pair kernel instantiations (alphabets of <= 4 symbols).
#include "ga_launch.h"
#include "ga_longpk.cuh"

namespace ga {

#define GA_KW_DEFINE(NAME, MODE)                                                      \
  cudaError_t launch_##NAME(const KBParams &p, int grid, cudaStream_t s) {            \
    kw_kernel<MODE, kKwK><<<grid, kKbThreads, 0, s>>>(p);                              \
    return cudaGetLastError();                                                         \
  }                                                                                    \
  int blocks_per_sm_##NAME() {                                                         \
    int n = 0;                                                                         \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kw_kernel<MODE, kKwK>, kKbThreads, 0); \
    return n;                                                                          \
  }

GA_KW_DEFINE(kw_local, kModeLocal)
GA_KW_DEFINE(kw_global, kModeGlobal)
GA_KW_DEFINE(kw_semi, kModeSemi)

}  // namespace ga
