// issue_rate.cu -- issue-rate probes behind the ALU roofline of the
// alignment kernels (built as the benchmark's own libga_roofline.so).
//
// The roofline of the DP kernels is an integer-issue bound: GCUPS <=
// SMs x clock x (lane-ops per clock per SM) / (ops per cell), the paper's
// theoretical-peak form (Sec. 4.2, Eq. TPP, Table 2).  These kernels measure
// the lane-op rate of each operation the cell update uses on this GPU: every
// thread runs 8 independent dependency chains of one operation, so the rate
// is throughput-bound, not latency-bound.
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "issue_rate.h"

namespace {

__device__ __forceinline__ uint32_t prmt_g(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}

template <int OP>
__device__ __forceinline__ uint32_t op(uint32_t x, uint32_t y, uint32_t z) {
  if constexpr (OP == RL_PROBE_VADD2) return __vadd2(x, y);
  if constexpr (OP == RL_PROBE_VMAXS2) return __vmaxs2(x, y);
  if constexpr (OP == RL_PROBE_VIADDMAX_S16X2) return __viaddmax_s16x2(x, y, z);
  if constexpr (OP == RL_PROBE_VIMAX3_S16X2) return __vimax3_s16x2(x, y, z);
  if constexpr (OP == RL_PROBE_VIADDMAX_S16X2_RELU) return __viaddmax_s16x2_relu(x, y, z);
  if constexpr (OP == RL_PROBE_PRMT) return prmt_g(x, y, z);
  if constexpr (OP == RL_PROBE_IADD) return x + y;
  if constexpr (OP == RL_PROBE_IMAX) return (uint32_t)max((int)x, (int)y);
  if constexpr (OP == RL_PROBE_VIADDMAX_S32) return (uint32_t)__viaddmax_s32((int)x, (int)y, (int)z);
  if constexpr (OP == RL_PROBE_VIMAX3_S32) return (uint32_t)__vimax3_s32((int)x, (int)y, (int)z);
  if constexpr (OP == RL_PROBE_IMAD) return x * y + z;
  if constexpr (OP == RL_PROBE_LOP3) return (x & y) | (z ^ y);
  if constexpr (OP == RL_PROBE_HADD2) {
    __half2 a = *reinterpret_cast<__half2 *>(&x), b = *reinterpret_cast<__half2 *>(&y);
    __half2 r = __hadd2(a, b);
    return *reinterpret_cast<uint32_t *>(&r);
  }
  if constexpr (OP == RL_PROBE_HMAX2) {
    __half2 a = *reinterpret_cast<__half2 *>(&x), b = *reinterpret_cast<__half2 *>(&y);
    __half2 r = __hmax2(a, b);
    return *reinterpret_cast<uint32_t *>(&r);
  }
  return x;
}

template <int OP>
__global__ void probe_kernel(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed * (threadIdx.x + 17 * k + 1);
  const uint32_t z = seed ^ 0x5410u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      // each step reads the neighbouring chain's previous value, so no
      // operand is loop-invariant and nothing can be folded or hoisted;
      // the 8 updates of a step are still independent of each other
      uint32_t b[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) b[k] = a[(k + 1) & 7];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = op<OP>(a[k], b[k], z);
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= a[k];
  if (s == 0x12345678u) sink[threadIdx.x] = s;  // keeps the chains alive
}

// The cell update of the inter-sequence kernel as a throughput probe, 8
// independent columns per thread: per column the substitution score by a
// byte permute, the diagonal add, the 3-way max of Eq. H, H - alpha and
// the fused add-max updates of Eqs. E and F (the F chain runs through the
// columns, as in the kernel).  S32 selects int32 cells.
template <bool S32>
__global__ void probe_mix_kernel(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t H[8], E[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    H[k] = seed * (threadIdx.x + k + 1);
    E[k] = seed ^ (k * 77u);
  }
  uint32_t F = seed, tw0 = seed * 3u, tw1 = seed * 5u;
  const uint32_t NA = S32 ? (uint32_t)-5 : 0xfffbfffbu, NB = S32 ? (uint32_t)-2 : 0xfffefffeu;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t sg = prmt_g(tw0, tw1, 0x5410u + (uint32_t)k);
        const uint32_t hd = H[(k + 7) & 7];
        if constexpr (S32) {
          const int d = (int)hd + (int)sg;
          const int h = __vimax3_s32(d, (int)E[k], (int)F);
          const int A = h + (int)NA;
          E[k] = (uint32_t)__viaddmax_s32((int)E[k], (int)NB, A);
          F = (uint32_t)__viaddmax_s32((int)F, (int)NB, A);
          H[k] = (uint32_t)h;
        } else {
          const uint32_t d = __vadd2(hd, sg);
          const uint32_t h = __vimax3_s16x2(d, E[k], F);
          const uint32_t A = __vadd2(h, NA);
          E[k] = __viaddmax_s16x2(E[k], NB, A);
          F = __viaddmax_s16x2(F, NB, A);
          H[k] = h;
        }
      }
      tw0 += 1;
    }
  }
  uint32_t s = F;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= H[k] ^ E[k];
  if (s == 0x12345678u) sink[threadIdx.x] = s;
}

template <int OP>
cudaError_t run(int iters, int blocks, int threads, uint32_t *sink, cudaStream_t s) {
  probe_kernel<OP><<<blocks, threads, 0, s>>>(iters, 0x9e3779b9u, sink);
  return cudaGetLastError();
}

}  // namespace

extern "C" int rl_issue_rate(int which, int iters, int blocks, int threads, float *ms,
                                   double *lane_ops) {
  if (!ms || !lane_ops || iters <= 0 || blocks <= 0 || threads <= 0 || threads > 1024 ||
      (threads & 31))
    return 1;
  uint32_t *sink = nullptr;
  if (cudaMalloc(&sink, 4096 * sizeof(uint32_t)) != cudaSuccess) return 3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaSuccess;
  auto launch = [&]() -> cudaError_t {
    switch (which) {
      case RL_PROBE_VADD2: return run<RL_PROBE_VADD2>(iters, blocks, threads, sink, 0);
      case RL_PROBE_VMAXS2: return run<RL_PROBE_VMAXS2>(iters, blocks, threads, sink, 0);
      case RL_PROBE_VIADDMAX_S16X2: return run<RL_PROBE_VIADDMAX_S16X2>(iters, blocks, threads, sink, 0);
      case RL_PROBE_VIMAX3_S16X2: return run<RL_PROBE_VIMAX3_S16X2>(iters, blocks, threads, sink, 0);
      case RL_PROBE_VIADDMAX_S16X2_RELU: return run<RL_PROBE_VIADDMAX_S16X2_RELU>(iters, blocks, threads, sink, 0);
      case RL_PROBE_PRMT: return run<RL_PROBE_PRMT>(iters, blocks, threads, sink, 0);
      case RL_PROBE_IADD: return run<RL_PROBE_IADD>(iters, blocks, threads, sink, 0);
      case RL_PROBE_IMAX: return run<RL_PROBE_IMAX>(iters, blocks, threads, sink, 0);
      case RL_PROBE_VIADDMAX_S32: return run<RL_PROBE_VIADDMAX_S32>(iters, blocks, threads, sink, 0);
      case RL_PROBE_VIMAX3_S32: return run<RL_PROBE_VIMAX3_S32>(iters, blocks, threads, sink, 0);
      case RL_PROBE_IMAD: return run<RL_PROBE_IMAD>(iters, blocks, threads, sink, 0);
      case RL_PROBE_LOP3: return run<RL_PROBE_LOP3>(iters, blocks, threads, sink, 0);
      case RL_PROBE_HADD2: return run<RL_PROBE_HADD2>(iters, blocks, threads, sink, 0);
      case RL_PROBE_HMAX2: return run<RL_PROBE_HMAX2>(iters, blocks, threads, sink, 0);
      case RL_PROBE_MIX_KA:
        probe_mix_kernel<false><<<blocks, threads>>>(iters, 0x9e3779b9u, sink);
        return cudaGetLastError();
      case RL_PROBE_MIX_S32:
        probe_mix_kernel<true><<<blocks, threads>>>(iters, 0x9e3779b9u, sink);
        return cudaGetLastError();
      default: return cudaErrorInvalidValue;
    }
  };
  err = launch();  // warm-up
  if (err == cudaSuccess) {
    cudaEventRecord(e0);
    err = launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
  }
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return 4;
  *ms = t;
  // operations per thread: iters * 16 * 8 (the mix probes count 6 ops per column)
  const bool mix = which == RL_PROBE_MIX_KA || which == RL_PROBE_MIX_S32;
  const double per_thread = (double)iters * 16.0 * 8.0 * (mix ? 6.0 : 1.0);
  *lane_ops = per_thread * (double)blocks * (double)threads;
  return 0;
}
