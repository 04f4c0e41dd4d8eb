// ga_probe.cu -- issue-rate probes behind the ALU roofline.
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

#include "../../include/gotoh_probe.h"

namespace {

__device__ __forceinline__ uint32_t prmt_g(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}

template <int OP>
__device__ __forceinline__ uint32_t op(uint32_t x, uint32_t y, uint32_t z) {
  if constexpr (OP == GA_PROBE_VADD2) return __vadd2(x, y);
  if constexpr (OP == GA_PROBE_VMAXS2) return __vmaxs2(x, y);
  if constexpr (OP == GA_PROBE_VIADDMAX_S16X2) return __viaddmax_s16x2(x, y, z);
  if constexpr (OP == GA_PROBE_VIMAX3_S16X2) return __vimax3_s16x2(x, y, z);
  if constexpr (OP == GA_PROBE_VIADDMAX_S16X2_RELU) return __viaddmax_s16x2_relu(x, y, z);
  if constexpr (OP == GA_PROBE_PRMT) return prmt_g(x, y, z);
  if constexpr (OP == GA_PROBE_IADD) return x + y;
  if constexpr (OP == GA_PROBE_IMAX) return (uint32_t)max((int)x, (int)y);
  if constexpr (OP == GA_PROBE_VIADDMAX_S32) return (uint32_t)__viaddmax_s32((int)x, (int)y, (int)z);
  if constexpr (OP == GA_PROBE_VIMAX3_S32) return (uint32_t)__vimax3_s32((int)x, (int)y, (int)z);
  if constexpr (OP == GA_PROBE_IMAD) return x * y + z;
  if constexpr (OP == GA_PROBE_LOP3) return (x & y) | (z ^ y);
  if constexpr (OP == GA_PROBE_HADD2) {
    __half2 a = *reinterpret_cast<__half2 *>(&x), b = *reinterpret_cast<__half2 *>(&y);
    __half2 r = __hadd2(a, b);
    return *reinterpret_cast<uint32_t *>(&r);
  }
  if constexpr (OP == GA_PROBE_HMAX2) {
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

// The cell update of one packed column (prmt, then 5 DPX/SIMD ops) as a
// throughput probe: 8 independent columns per thread.
__global__ void probe_cell_kernel(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t H[8], E[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    H[k] = seed * (threadIdx.x + k + 1);
    E[k] = seed ^ (k * 77u);
  }
  uint32_t F = seed, tw0 = seed * 3u, tw1 = seed * 5u;
  const uint32_t NA = 0xfffbfffbu, NB = 0xfffefffeu, sel = 0x5410u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint32_t sg = prmt_g(tw0, tw1, sel + k);
        uint32_t d = __viaddmax_s16x2(H[k], sg, E[k]);
        uint32_t h = __vmaxs2(d, F);
        uint32_t A = __vadd2(h, NA);
        E[k] = __viaddmax_s16x2(E[k], NB, A);
        F = __viaddmax_s16x2(F, NB, A) ^ (uint32_t)k;
        H[k] = h;
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

extern "C" int ga_probe_issue_rate(int which, int iters, int blocks, int threads, float *ms,
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
      case GA_PROBE_VADD2: return run<GA_PROBE_VADD2>(iters, blocks, threads, sink, 0);
      case GA_PROBE_VMAXS2: return run<GA_PROBE_VMAXS2>(iters, blocks, threads, sink, 0);
      case GA_PROBE_VIADDMAX_S16X2: return run<GA_PROBE_VIADDMAX_S16X2>(iters, blocks, threads, sink, 0);
      case GA_PROBE_VIMAX3_S16X2: return run<GA_PROBE_VIMAX3_S16X2>(iters, blocks, threads, sink, 0);
      case GA_PROBE_VIADDMAX_S16X2_RELU: return run<GA_PROBE_VIADDMAX_S16X2_RELU>(iters, blocks, threads, sink, 0);
      case GA_PROBE_PRMT: return run<GA_PROBE_PRMT>(iters, blocks, threads, sink, 0);
      case GA_PROBE_IADD: return run<GA_PROBE_IADD>(iters, blocks, threads, sink, 0);
      case GA_PROBE_IMAX: return run<GA_PROBE_IMAX>(iters, blocks, threads, sink, 0);
      case GA_PROBE_VIADDMAX_S32: return run<GA_PROBE_VIADDMAX_S32>(iters, blocks, threads, sink, 0);
      case GA_PROBE_VIMAX3_S32: return run<GA_PROBE_VIMAX3_S32>(iters, blocks, threads, sink, 0);
      case GA_PROBE_IMAD: return run<GA_PROBE_IMAD>(iters, blocks, threads, sink, 0);
      case GA_PROBE_LOP3: return run<GA_PROBE_LOP3>(iters, blocks, threads, sink, 0);
      case GA_PROBE_HADD2: return run<GA_PROBE_HADD2>(iters, blocks, threads, sink, 0);
      case GA_PROBE_HMAX2: return run<GA_PROBE_HMAX2>(iters, blocks, threads, sink, 0);
      case GA_PROBE_CELL:
        probe_cell_kernel<<<blocks, threads>>>(iters, 0x9e3779b9u, sink);
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
  // operations per thread: iters * 16 * 8 (the cell probe counts its 6 ops)
  const double per_thread = (double)iters * 16.0 * 8.0 * (which == GA_PROBE_CELL ? 6.0 : 1.0);
  *lane_ops = per_thread * (double)blocks * (double)threads;
  return 0;
}
