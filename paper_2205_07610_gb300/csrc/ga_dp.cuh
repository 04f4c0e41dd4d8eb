// ga_dp.cuh -- the register-tiled row update shared by every DP kernel.
//
// One lane owns K adjacent columns j0..j0+K-1 of the DP matrix in registers
// (Sec. 3.1, register tiling with "unrolled arrays", Sec. 3.2).  For row i
// it receives from its left neighbour H(i, j0-1) folded into F(i, j0)
// (Fin) and the diagonal H(i-1, j0-1) (Hdiag), and updates in place:
//
//   pass 1 (right to left):  H_j <- H_{j-1} + sigma(i, j)    (H_{j-1} still
//                                                             holds row i-1)
//   pass 2 (left to right):  H_j <- max(H_j, E_j, F)         (Eq. H; local
//                                                             mode also 0)
//                            A   <- H_j - alpha
//                            E_j <- max(E_j - beta, A)       (Eq. E, row i+1)
//                            F   <- max(F - beta, A)         (Eq. F, col j+1)
//
// Pipe balance on sm_103a: the packed add runs on the FMA pipe, the max /
// fused add-max / byte-permute ops on the ALU pipe, each at 16 lanes per
// clock per SM sub-partition.  Per register this is 2 FMA-pipe ops (the two
// adds) and 4 ALU-pipe ops (3-way max, two fused add-max, the sigma prmt),
// against the 7 scalar ops per cell of the paper's count (Sec. 4.2).  On
// exit H holds row i, E holds E(i+1, .), and the returned F is F(i, j0+K)
// for the right neighbour.
#pragma once

#include <type_traits>

#include "ga_common.cuh"

namespace ga {

// Byte permute, PTX generic mode: the msb of each selector nibble
// replicates the sign of the selected byte (used to sign-extend int8
// substitution scores and to produce sigma in {0,-1} for pad columns).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

template <class Cell>
struct CellInfo {
  static constexpr bool kPacked = !std::is_same<typename Cell::T, int32_t>::value;
  static constexpr int kHalves = kPacked ? 2 : 1;
  static constexpr int kNeg = kPacked ? kNeg16 : kNeg32;
};

// Selector that turns byte b of word a (and, packed, byte b of word c into
// the high half) into a sign-extended cell value.
template <class Cell>
__host__ __device__ constexpr uint32_t sext_sel(int b) {
  return CellInfo<Cell>::kPacked
             ? (uint32_t)(b | ((b | 8) << 4) | ((b + 4) << 8) | ((b + 12) << 12))
             : (uint32_t)(b | ((b | 8) << 4) | ((b | 8) << 8) | ((b | 8) << 12));
}

// The row update.  SIG(j) returns the (packed) substitution score of
// column j for this row; NA(j) the (packed) -alpha of column j (the
// semi-global kernel frees the gaps leaving the last real column).
template <class Cell, int MODE, int K, class SigFn, class NaFn>
__device__ __forceinline__ typename Cell::T dp_row(typename Cell::T (&H)[K], typename Cell::T (&E)[K],
                                                    typename Cell::T Hdiag, typename Cell::T Fin,
                                                    typename Cell::T NB, typename Cell::T &best,
                                                    SigFn SIG, NaFn NA) {
  using T = typename Cell::T;
#pragma unroll
  for (int j = K - 1; j >= 1; --j) H[j] = Cell::add(H[j - 1], SIG(j));
  H[0] = Cell::add(Hdiag, SIG(0));
  T F = Fin;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    H[j] = (MODE == kModeLocal) ? Cell::max3_relu(H[j], E[j], F) : Cell::max3(H[j], E[j], F);
    T A = Cell::add(H[j], NA(j));
    E[j] = Cell::addmax(E[j], NB, A);
    F = Cell::addmax(F, NB, A);
    if constexpr (MODE == kModeLocal) {
      if ((j & 1) == 1) best = Cell::max3(best, H[j - 1], H[j]);
      else if (j == K - 1) best = Cell::max(best, H[j]);
    }
  }
  return F;
}

// Extract half h of a cell as int.
template <class Cell>
__device__ __forceinline__ int cell_get(typename Cell::T v, int h) {
  if constexpr (CellInfo<Cell>::kPacked) return h ? hi16((uint32_t)v) : lo16((uint32_t)v);
  else return (int)v;
}

// Warp-reduce max within groups of G lanes.
template <int G>
__device__ __forceinline__ int group_max(int v) {
#pragma unroll
  for (int off = G / 2; off >= 1; off >>= 1) v = ::max(v, __shfl_xor_sync(0xffffffffu, v, off, G));
  return v;
}

// 2-bit code of the residue at position pos of a flat packed stream
// (residue x of the code buffer lives in word x / 16, bits 2*(x % 16)).
__device__ __forceinline__ int packed_code(const uint32_t *base, int64_t pos) {
  const uint32_t w = __ldg(base + (pos >> 4));
  return (int)((w >> (2 * (int)(pos & 15))) & 3u);
}

}  // namespace ga
