// ga_mlp.cuh -- the band predictor's network on the GPU (not part of the
// paper): 32 pair features -> relu(64) -> relu(64) -> y = log2(1 + w), with
// bf16 weights and float32 arithmetic.
//
// Parameter vector (float32 master / bf16 copy), row-major, in this order:
//   W1[64][32], b1[64], W2[64][64], b2[64], w3[64], b3   (6337 values)
// Loss of a batch of B samples with targets t: L = sum_b (y_b - t_b)^2 / (2B).
//
// This header holds the layout and the per-unit arithmetic shared by the
// training kernels (ga_mlp.cu) and the fused predictor (ga_band.cuh).
#pragma once

#include <cstdint>

namespace ga {

constexpr int kMlpIn = 32, kMlpH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn, kOffW2 = kOffB1 + kMlpH,
              kOffB2 = kOffW2 + kMlpH * kMlpH, kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpH;
constexpr int kMlpParams = kOffB3 + 1;  // 6337
constexpr int kMlpParamsPadded = (kMlpParams + 3) & ~3;
// Per-sample scratch row: x, h1, d1 (dL/dz1), h2, d2 (dL/dz2), dy, r.
constexpr int kSX = 0, kSH1 = kSX + kMlpIn, kSD1 = kSH1 + kMlpH, kSH2 = kSD1 + kMlpH,
              kSD2 = kSH2 + kMlpH, kSDY = kSD2 + kMlpH, kSR = kSDY + 1;
constexpr int kScratchRow = 292;  // >= kSR + 1, multiple of 4
static_assert(kMlpParams == 6337, "parameter layout");
static_assert(kScratchRow >= kSR + 1, "scratch row");

__device__ __forceinline__ float bf16_bits_to_f32(uint16_t b) {
  return __uint_as_float((uint32_t)b << 16);
}

// Round to nearest even of a finite float32 to bf16 (NaN stays a quiet NaN).
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (uint16_t)((u >> 16) | 0x40u);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// Stage the bf16 parameters as float in shared memory (whole block).
__device__ __forceinline__ void stage_params(const uint16_t *__restrict__ wb, float *ws) {
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) ws[k] = bf16_bits_to_f32(wb[k]);
}

// Hidden unit o of layer 1 / layer 2 and the output, each a dot product in
// index order (the same order in every kernel, so that every kernel gives
// the same float32 result for the same sample).  Activations are read with
// a stride (thread-private columns of a shared-memory array, or contiguous).
__device__ __forceinline__ float unit1(const float *ws, int o, const float *x, int xs) {
  float z = ws[kOffB1 + o];
#pragma unroll 8
  for (int i = 0; i < kMlpIn; ++i) z = fmaf(ws[kOffW1 + o * kMlpIn + i], x[i * xs], z);
  return z;
}
// Layer-2 unit from the layer-1 pre-activations z1 (relu applied on the fly).
__device__ __forceinline__ float unit2(const float *ws, int o, const float *z1, int zs) {
  float z = ws[kOffB2 + o];
#pragma unroll 8
  for (int i = 0; i < kMlpH; ++i) z = fmaf(ws[kOffW2 + o * kMlpH + i], fmaxf(z1[i * zs], 0.f), z);
  return z;
}
__device__ __forceinline__ float output(const float *ws, const float *h2, int hs) {
  float y = ws[kOffB3];
#pragma unroll 8
  for (int o = 0; o < kMlpH; ++o) y = fmaf(ws[kOffW3 + o], h2[o * hs], y);
  return y;
}

}  // namespace ga
