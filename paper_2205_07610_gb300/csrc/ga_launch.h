// ga_launch.h -- host-side launchers of the templated DP kernels.  Each
// instantiation family lives in its own translation unit so the library
// compiles in parallel.
#pragma once

#include <cuda_runtime.h>

#include "ga_inter.cuh"
#include "ga_long.cuh"

namespace ga {

// Column tile per lane of the inter-sequence bins; a group has 16 lanes, so
// bin b covers pairs whose shorter sequence has at most 16 * kKaK[b] residues.
constexpr int kKaG = 16;
constexpr int kKaNumBins = 9;
constexpr int kKaK[kKaNumBins] = {8, 10, 12, 14, 16, 18, 20, 24, 32};
constexpr int kKaThreads = 128;

// Long kernel: 32 lanes x 16 columns per stage.
constexpr int kKbK = 16;
// Banded kernel: 32 lanes x 16 columns per stage, 16-column band blocks.
constexpr int kKcK = 16;
constexpr int kKcThreads = 128;
constexpr int kKcWarps = kKcThreads / 32;
constexpr int kKbThreads = 128;
constexpr int kKbWarps = kKbThreads / 32;

// One launcher / occupancy query per (cell type, mode) and per mode and
// substitution path of the long kernel; defined in ga_ka*_*.cu and ga_kb.cu.
#define GA_KA_DECLARE(NAME)                                                          \
  cudaError_t launch_##NAME(int bin, const KAParams &p, int grid, cudaStream_t s);  \
  int blocks_per_sm_##NAME(int bin);
GA_KA_DECLARE(ka16_local)
GA_KA_DECLARE(ka16_global)
GA_KA_DECLARE(ka16_semi)
GA_KA_DECLARE(ka32_local)
GA_KA_DECLARE(ka32_global)
GA_KA_DECLARE(ka32_semi)

#define GA_KB_DECLARE(NAME)                                                                 \
  cudaError_t launch_##NAME(const KBParams &p, int grid, size_t smem, cudaStream_t s);     \
  int blocks_per_sm_##NAME(size_t smem);
GA_KB_DECLARE(kb_local_sel)
GA_KB_DECLARE(kb_global_sel)
GA_KB_DECLARE(kb_semi_sel)
GA_KB_DECLARE(kb_local_prof)
GA_KB_DECLARE(kb_global_prof)
GA_KB_DECLARE(kb_semi_prof)

struct KCParams;
cudaError_t launch_kc(const KCParams &p, int grid, cudaStream_t s);
int blocks_per_sm_kc();

#define GA_KA_OCC(CELL, MODE, K)                                                             \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ka_kernel<CELL, MODE, kKaG, K>, kKaThreads, 0)

#define GA_KA_DEFINE(NAME, CELL, MODE)                                                         \
  cudaError_t launch_##NAME(int bin, const KAParams &p, int grid, cudaStream_t s) {            \
    switch (bin) {                                                                             \
      case 0: ka_kernel<CELL, MODE, kKaG, 8><<<grid, kKaThreads, 0, s>>>(p); break;            \
      case 1: ka_kernel<CELL, MODE, kKaG, 10><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 2: ka_kernel<CELL, MODE, kKaG, 12><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 3: ka_kernel<CELL, MODE, kKaG, 14><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 4: ka_kernel<CELL, MODE, kKaG, 16><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 5: ka_kernel<CELL, MODE, kKaG, 18><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 6: ka_kernel<CELL, MODE, kKaG, 20><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 7: ka_kernel<CELL, MODE, kKaG, 24><<<grid, kKaThreads, 0, s>>>(p); break;           \
      case 8: ka_kernel<CELL, MODE, kKaG, 32><<<grid, kKaThreads, 0, s>>>(p); break;           \
      default: return cudaErrorInvalidValue;                                                   \
    }                                                                                          \
    return cudaGetLastError();                                                                 \
  }                                                                                            \
  int blocks_per_sm_##NAME(int bin) {                                                          \
    int n = 0;                                                                                 \
    switch (bin) {                                                                             \
      case 0: GA_KA_OCC(CELL, MODE, 8); break;                                                 \
      case 1: GA_KA_OCC(CELL, MODE, 10); break;                                                \
      case 2: GA_KA_OCC(CELL, MODE, 12); break;                                                \
      case 3: GA_KA_OCC(CELL, MODE, 14); break;                                                \
      case 4: GA_KA_OCC(CELL, MODE, 16); break;                                                \
      case 5: GA_KA_OCC(CELL, MODE, 18); break;                                                \
      case 6: GA_KA_OCC(CELL, MODE, 20); break;                                                \
      case 7: GA_KA_OCC(CELL, MODE, 24); break;                                                \
      case 8: GA_KA_OCC(CELL, MODE, 32); break;                                                \
      default: break;                                                                          \
    }                                                                                          \
    return n;                                                                                  \
  }

#define GA_KB_DEFINE(NAME, MODE, PROFILE)                                                    \
  cudaError_t launch_##NAME(const KBParams &p, int grid, size_t smem, cudaStream_t s) {     \
    if (smem > 48 * 1024) {                                                                  \
      cudaError_t e = cudaFuncSetAttribute(kb_kernel<MODE, kKbK, PROFILE>,                   \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                           (int)smem);                                       \
      if (e != cudaSuccess) return e;                                                        \
    }                                                                                        \
    kb_kernel<MODE, kKbK, PROFILE><<<grid, kKbThreads, smem, s>>>(p);                        \
    return cudaGetLastError();                                                               \
  }                                                                                          \
  int blocks_per_sm_##NAME(size_t smem) {                                                    \
    int n = 0;                                                                               \
    if (smem > 48 * 1024)                                                                    \
      cudaFuncSetAttribute(kb_kernel<MODE, kKbK, PROFILE>,                                   \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_kernel<MODE, kKbK, PROFILE>,        \
                                                  kKbThreads, smem);                         \
    return n;                                                                                \
  }

}  // namespace ga
