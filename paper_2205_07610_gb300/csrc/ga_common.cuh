// ga_common.cuh -- shared device definitions for the Gotoh alignment kernels.
//
// Cell arithmetic follows Eqs. H, E, F of Sec. 2.1 (AnySeq/GPU, ICS'22).
// Two cell types are used:
//   * packed int16x2: two independent alignments in the low / high halves
//     of one 32-bit register (the paper's half2 packing, Sec. 3.2, made
//     exact with integer SIMD instead of fp16);
//   * int32: one alignment per register.
// The fused Blackwell DPX operations (max(a+b, c), max(a,b,c), with and
// without a ReLU clamp at 0) evaluate the recurrence in 5 fused ops per
// cell instead of the 7 scalar ops of the paper's count (Sec. 4.2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gotoh_align.h"

namespace ga {

constexpr int kModeLocal = GA_LOCAL;
constexpr int kModeGlobal = GA_GLOBAL;
constexpr int kModeSemi = GA_SEMIGLOBAL;

// -inf sentinels.  int16: -32000 leaves room for one further gap cost
// (beta <= 700 on the int16 path) without wrapping.  int32: far below any
// admitted score (|score| < 2^30).
constexpr int kNeg16 = -32000;
constexpr int kNeg32 = -(1 << 30) - (1 << 29);
constexpr int kInt16Bound = 30000;  // |reachable value| bound for int16 routing
constexpr int kInt16MaxGap = 700;   // alpha, beta limit for int16 routing

// Per-pair classes written by the planning kernel.
enum PairClass : uint32_t {
  kClassInter16 = 0,   // packed int16x2 inter-sequence kernel
  kClassInter32 = 1,   // int32 inter-sequence kernel
  kClassLong = 2,      // intra-sequence (long / large-alphabet) kernel
  kClassDone = 3,      // trivial or invalid: score written by the planner
};

__device__ __forceinline__ uint32_t pack2(int lo, int hi) {
  return (uint32_t)(lo & 0xffff) | ((uint32_t)hi << 16);
}
__device__ __forceinline__ uint32_t splat2(int v) { return pack2(v, v); }
__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xffff); }
__device__ __forceinline__ int hi16(uint32_t v) { return (int)(int16_t)(v >> 16); }

// ---- cell operations ---------------------------------------------------
struct CellS16x2 {
  using T = uint32_t;
  static __device__ __forceinline__ T add(T a, T b) { return __vadd2(a, b); }
  static __device__ __forceinline__ T max(T a, T b) { return __vmaxs2(a, b); }
  static __device__ __forceinline__ T addmax(T a, T b, T c) { return __viaddmax_s16x2(a, b, c); }
  static __device__ __forceinline__ T addmax_relu(T a, T b, T c) {
    return __viaddmax_s16x2_relu(a, b, c);
  }
  static __device__ __forceinline__ T max3(T a, T b, T c) { return __vimax3_s16x2(a, b, c); }
  static __device__ __forceinline__ T max3_relu(T a, T b, T c) { return __vimax3_s16x2_relu(a, b, c); }
  static __device__ __forceinline__ T splat(int v) { return splat2(v); }
};

struct CellS32 {
  using T = int32_t;
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T max(T a, T b) { return ::max(a, b); }
  static __device__ __forceinline__ T addmax(T a, T b, T c) { return __viaddmax_s32(a, b, c); }
  static __device__ __forceinline__ T addmax_relu(T a, T b, T c) {
    return __viaddmax_s32_relu(a, b, c);
  }
  static __device__ __forceinline__ T max3(T a, T b, T c) { return __vimax3_s32(a, b, c); }
  static __device__ __forceinline__ T max3_relu(T a, T b, T c) { return __vimax3_s32_relu(a, b, c); }
  static __device__ __forceinline__ T splat(int v) { return v; }
};

// Device status word helpers: first error wins.
__device__ __forceinline__ void set_status(int32_t *status, int code) {
  if (status) atomicCAS(status, 0, code);
}

}  // namespace ga
