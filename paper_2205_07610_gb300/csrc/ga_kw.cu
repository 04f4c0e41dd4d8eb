// Packed int16x2 long-pair kernel instantiations (alphabets of <= 4 symbols).
#include "ga_launch.h"
#include "ga_longpk.cuh"

namespace ga {

#define GA_KW_DEFINE(NAME, MODE, K)                                                   \
  cudaError_t launch_##NAME(const KBParams &p, int grid, cudaStream_t s) {            \
    kw_kernel<MODE, K><<<grid, kKbThreads, 0, s>>>(p);                                 \
    return cudaGetLastError();                                                         \
  }                                                                                    \
  int blocks_per_sm_##NAME() {                                                         \
    int n = 0;                                                                         \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kw_kernel<MODE, K>, kKbThreads, 0); \
    return n;                                                                          \
  }

GA_KW_DEFINE(kw_local, kModeLocal, kKwKLocal)
GA_KW_DEFINE(kw_global, kModeGlobal, kKwKGlobal)
GA_KW_DEFINE(kw_semi, kModeSemi, kKwKSemi)

}  // namespace ga
