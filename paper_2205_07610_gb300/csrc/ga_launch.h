// ga_launch.h -- host-side launchers of the templated DP kernels.  Each
// instantiation family lives in its own translation unit so the library
// compiles in parallel.
#pragma once

#include <cuda_runtime.h>

#include "ga_inter.cuh"
#include "ga_long.cuh"
#include "ga_longpk.cuh"
#include "ga_bandcz.cuh"

namespace ga {

// Lanes per pair of the inter-sequence bins: bin b covers pairs whose
// shorter sequence has at most 16 * kKaK[b] residues (kKaK in ga_inter.cuh).
constexpr int kKaG = 16;
constexpr int kKaThreads = 128;

// Long kernel: 32 lanes x 16 columns per stage.
constexpr int kKbK = 16;
// Banded kernel: 32 lanes x 16 columns per stage, 16-column band blocks.
constexpr int kKcK = 16;
constexpr int kKcThreads = 128;
constexpr int kKcWarps = kKcThreads / 32;
// Columns of a super-stage of the packed band kernel (64 blocks of kKcK
// columns): the unit of the band order's work key.
constexpr int kBandStageCols = 64 * kKcK;
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

// Alternative lane-group size of the packed int16x2 tiles, same tile width
// (16 x kKaK[b] columns): tiles 0..6 (K = 6..12) also run with 8 lanes x 2K
// columns per pair (half the wavefront fill, twice the registers per lane),
// tiles 10, 12, 14, 15, 16 (K = 16, 18, 20, 24, 32) with 32 lanes x K/2
// columns (fewer registers, twice the fill).  A plan's tuning picks per tile.
constexpr int ka_alt_g(int bin) {
  return bin <= 6 ? 8 : (bin >= 10 && kKaK[bin] % 2 == 0) ? 32 : 0;
}
constexpr int ka_alt_k(int bin) {
  return ka_alt_g(bin) == 8 ? 2 * kKaK[bin] : ka_alt_g(bin) == 32 ? kKaK[bin] / 2 : 0;
}
constexpr uint32_t ka_alt_mask() {
  uint32_t m = 0;
  for (int b = 0; b < kKaNumBins; ++b)
    if (ka_alt_g(b)) m |= 1u << b;
  return m;
}
constexpr uint32_t kKaAltTiles = ka_alt_mask();
GA_KA_DECLARE(ka16alt_local)
GA_KA_DECLARE(ka16alt_global)
GA_KA_DECLARE(ka16alt_semi)

#define GA_KB_DECLARE(NAME)                                                                 \
  cudaError_t launch_##NAME(const KBParams &p, int grid, size_t smem, cudaStream_t s);     \
  int blocks_per_sm_##NAME(size_t smem);
GA_KB_DECLARE(kb_local_sel)
GA_KB_DECLARE(kb_global_sel)
GA_KB_DECLARE(kb_semi_sel)
GA_KB_DECLARE(kb_local_prof)
GA_KB_DECLARE(kb_global_prof)
GA_KB_DECLARE(kb_semi_prof)

// Packed long kernel (alphabets of <= 4 symbols, sigma_max + alpha <=
// kKwMaxStep): 32 lanes x K columns per half, two halves per super-stage.
// K per mode as measured on GB300 on the 20k long DNA pairs (K = 8, 12, 16,
// 20, 24): 24 for local and global, 20 for semi-global.
constexpr int kKwKLocal = 24;
constexpr int kKwKGlobal = 24;
constexpr int kKwKSemi = 20;
cudaError_t launch_kw_local(const KBParams &p, int grid, cudaStream_t s);
cudaError_t launch_kw_global(const KBParams &p, int grid, cudaStream_t s);
cudaError_t launch_kw_semi(const KBParams &p, int grid, cudaStream_t s);
int blocks_per_sm_kw_local();
int blocks_per_sm_kw_global();
int blocks_per_sm_kw_semi();

struct KCParams;
cudaError_t launch_kc(const KCParams &p, int grid, cudaStream_t s);
int blocks_per_sm_kc();
// Packed banded kernel (sigma_max + alpha <= kKzMaxStep, ga_bandcz.cuh);
// its edge buffer holds one KZEdge (16 bytes) per row and warp.
cudaError_t launch_kz(const KCParams &p, int grid, cudaStream_t s);
int blocks_per_sm_kz();

// Launch / occupancy of tile `bin` (compile-time recursion over the tiles).
template <class CELL, int MODE, int I = 0>
cudaError_t launch_ka_tile(int bin, const KAParams &p, int grid, cudaStream_t s) {
  if constexpr (I == kKaNumBins) {
    return cudaErrorInvalidValue;
  } else {
    if (bin == I) {
      ka_kernel<CELL, MODE, kKaG, kKaK[I]><<<grid, kKaThreads, 0, s>>>(p);
      return cudaGetLastError();
    }
    return launch_ka_tile<CELL, MODE, I + 1>(bin, p, grid, s);
  }
}

template <class CELL, int MODE, int I = 0>
int blocks_per_sm_ka_tile(int bin) {
  if constexpr (I == kKaNumBins) {
    return 0;
  } else {
    if (bin == I) {
      int n = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ka_kernel<CELL, MODE, kKaG, kKaK[I]>, kKaThreads, 0);
      return n;
    }
    return blocks_per_sm_ka_tile<CELL, MODE, I + 1>(bin);
  }
}

#define GA_KA_DEFINE(NAME, CELL, MODE)                                                  \
  cudaError_t launch_##NAME(int bin, const KAParams &p, int grid, cudaStream_t s) {     \
    return launch_ka_tile<CELL, MODE>(bin, p, grid, s);                                 \
  }                                                                                     \
  int blocks_per_sm_##NAME(int bin) { return blocks_per_sm_ka_tile<CELL, MODE>(bin); }

template <int MODE, int I = 0>
cudaError_t launch_ka_alt_tile(int bin, const KAParams &p, int grid, cudaStream_t s) {
  if constexpr (I == kKaNumBins) {
    return cudaErrorInvalidValue;
  } else {
    if (bin == I) {
      if constexpr (ka_alt_g(I) != 0) {
        ka_kernel<CellS16x2, MODE, ka_alt_g(I), ka_alt_k(I)><<<grid, kKaThreads, 0, s>>>(p);
        return cudaGetLastError();
      } else {
        return cudaErrorInvalidValue;
      }
    }
    return launch_ka_alt_tile<MODE, I + 1>(bin, p, grid, s);
  }
}

template <int MODE, int I = 0>
int blocks_per_sm_ka_alt_tile(int bin) {
  if constexpr (I == kKaNumBins) {
    return 0;
  } else {
    if (bin == I) {
      int n = 0;
      if constexpr (ka_alt_g(I) != 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ka_kernel<CellS16x2, MODE, ka_alt_g(I), ka_alt_k(I)>,
                                                      kKaThreads, 0);
      return n;
    }
    return blocks_per_sm_ka_alt_tile<MODE, I + 1>(bin);
  }
}

#define GA_KA_ALT_DEFINE(NAME, MODE)                                                    \
  cudaError_t launch_##NAME(int bin, const KAParams &p, int grid, cudaStream_t s) {     \
    return launch_ka_alt_tile<MODE>(bin, p, grid, s);                                   \
  }                                                                                     \
  int blocks_per_sm_##NAME(int bin) { return blocks_per_sm_ka_alt_tile<MODE>(bin); }

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
