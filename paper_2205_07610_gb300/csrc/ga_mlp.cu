// ga_mlp.cu -- training and inference kernels of the band predictor's
// network and their C ABI (include/gotoh_band.h).  Not part of the paper.
//
// A training step is two kernels:
//   mlp_fwd_bwd_kernel   : thread per batch sample; forward pass with the
//     bf16 weights (staged once per block in shared memory as float), then
//     the per-sample backward quantities, written to one scratch row each;
//   mlp_grad_adam_kernel : thread per parameter; its gradient is the sum
//     over the batch in sample order (deterministic, no atomics), then the
//     Adam update of the float32 master value and its bf16 copy.
// ga_mlp_train records its steps into a CUDA graph and launches that once.
#include <cmath>
#include <cstdio>

#include "../../include/gotoh_band.h"
#include "ga_common.cuh"
#include "ga_mlp.cuh"
#include "ga_pool.h"

namespace ga {

// Dynamic shared memory of the per-sample kernels: the parameters as float,
// then per thread two columns of 64 activations ([unit][thread] layout, so
// that a warp touches 32 consecutive words).
constexpr int kParamsPadded = kMlpParamsPadded;
__host__ __device__ constexpr size_t mlp_smem_bytes(int threads) {
  return sizeof(float) * ((size_t)kParamsPadded + 2 * (size_t)kMlpH * (size_t)threads);
}

// Thread per sample: y = net(x).  Inputs are rows of 32 floats.
__global__ void __launch_bounds__(128) mlp_forward_kernel(const uint16_t *__restrict__ wb,
                                                          const float *__restrict__ x, int64_t n,
                                                          float *__restrict__ y) {
  extern __shared__ float ws[];
  const int T = blockDim.x;
  float *a1 = ws + kParamsPadded + threadIdx.x, *a2 = a1 + kMlpH * T;
  stage_params(wb, ws);
  __syncthreads();
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    const float *xv = x + b * kMlpIn;
    for (int o = 0; o < kMlpH; ++o) a1[o * T] = unit1(ws, o, xv, 1);
    for (int o = 0; o < kMlpH; ++o) a2[o * T] = fmaxf(unit2(ws, o, a1, T), 0.f);
    y[b] = output(ws, a2, T);
  }
}

// Thread per batch sample: forward + per-sample backward into scratch rows.
// idx (nullable) maps batch position -> sample; inv_b = 1 / B.
__global__ void __launch_bounds__(128) mlp_fwd_bwd_kernel(const uint16_t *__restrict__ wb,
                                                          const float *__restrict__ x,
                                                          const float *__restrict__ target,
                                                          const int32_t *__restrict__ idx, int B,
                                                          int64_t nsamples, float inv_b,
                                                          float *__restrict__ scratch,
                                                          int32_t *__restrict__ status) {
  extern __shared__ float ws[];
  const int T = blockDim.x;
  float *a1 = ws + kParamsPadded + threadIdx.x, *a2 = a1 + kMlpH * T;
  stage_params(wb, ws);
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int64_t sample = idx ? (int64_t)idx[b] : (int64_t)b;
  float *row = scratch + (size_t)b * kScratchRow;
  if (sample < 0 || sample >= nsamples) {  // invalid batch index: zero row, error status
    for (int c = 0; c < kScratchRow; ++c) row[c] = 0.f;
    set_status(status, GA_ERR_ARG);
    return;
  }
  const float *xv = x + sample * kMlpIn;
  for (int i = 0; i < kMlpIn; ++i) row[kSX + i] = xv[i];
  for (int o = 0; o < kMlpH; ++o) {
    const float z = unit1(ws, o, xv, 1);
    a1[o * T] = z;  // pre-activation z1
    row[kSH1 + o] = fmaxf(z, 0.f);
  }
  for (int o = 0; o < kMlpH; ++o) {
    const float h = fmaxf(unit2(ws, o, a1, T), 0.f);
    a2[o * T] = h;
    row[kSH2 + o] = h;
  }
  const float y = output(ws, a2, T);
  const float r = y - target[sample];
  const float dy = r * inv_b;
  row[kSDY] = dy;
  row[kSR] = r;
  // d2 = dL/dz2 replaces h2 (z2 > 0 exactly where h2 > 0)
  for (int o = 0; o < kMlpH; ++o) {
    const float d = a2[o * T] > 0.f ? dy * ws[kOffW3 + o] : 0.f;
    a2[o * T] = d;
    row[kSD2 + o] = d;
  }
  // d1[i] = relu'(z1[i]) * sum_o d2[o] W2[o][i]
  for (int i = 0; i < kMlpH; ++i) {
    float acc = 0.f;
#pragma unroll 8
    for (int o = 0; o < kMlpH; ++o) acc = fmaf(a2[o * T], ws[kOffW2 + o * kMlpH + i], acc);
    row[kSD1 + i] = a1[i * T] > 0.f ? acc : 0.f;
  }
}

struct AdamArgs {
  float lr, beta1, beta2, eps;
  float c1, c2;  // 1 / (1 - beta1^t), 1 / (1 - beta2^t)
  int update;    // 0: gradient (and loss) only
};

// Thread per parameter (plus one for the loss): batch sums in sample order.
__global__ void __launch_bounds__(128) mlp_grad_adam_kernel(const float *__restrict__ scratch, int B,
                                                            float *__restrict__ master,
                                                            float *__restrict__ adam_m,
                                                            float *__restrict__ adam_v,
                                                            uint16_t *__restrict__ wb,
                                                            float *__restrict__ grad_out,
                                                            float *__restrict__ loss_out,
                                                            const AdamArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kMlpParams) return;
  if (k == kMlpParams) {  // loss
    if (loss_out) {
      float s = 0.f;
      for (int b = 0; b < B; ++b) {
        const float r = scratch[(size_t)b * kScratchRow + kSR];
        s = fmaf(r, r, s);
      }
      *loss_out = 0.5f * s / (float)B;
    }
    return;
  }
  int ua, ub;  // scratch columns multiplied: g = sum_b row[ua] * (ub < 0 ? 1 : row[ub])
  if (k < kOffB1) {
    ua = kSD1 + k / kMlpIn;
    ub = kSX + k % kMlpIn;
  } else if (k < kOffW2) {
    ua = kSD1 + (k - kOffB1);
    ub = -1;
  } else if (k < kOffB2) {
    ua = kSD2 + (k - kOffW2) / kMlpH;
    ub = kSH1 + (k - kOffW2) % kMlpH;
  } else if (k < kOffW3) {
    ua = kSD2 + (k - kOffB2);
    ub = -1;
  } else if (k < kOffB3) {
    ua = kSDY;
    ub = kSH2 + (k - kOffW3);
  } else {
    ua = kSDY;
    ub = -1;
  }
  float g = 0.f;
  if (ub >= 0) {
    for (int b = 0; b < B; ++b) {
      const float *row = scratch + (size_t)b * kScratchRow;
      g = fmaf(row[ua], row[ub], g);
    }
  } else {
    for (int b = 0; b < B; ++b) g += scratch[(size_t)b * kScratchRow + ua];
  }
  if (grad_out) grad_out[k] = g;
  if (!a.update) return;
  const float mk = fmaf(a.beta1, adam_m[k], (1.f - a.beta1) * g);
  const float vk = fmaf(a.beta2, adam_v[k], (1.f - a.beta2) * g * g);
  adam_m[k] = mk;
  adam_v[k] = vk;
  const float mhat = mk * a.c1, vhat = vk * a.c2;
  const float w = master[k] - a.lr * mhat / (sqrtf(vhat) + a.eps);
  master[k] = w;
  wb[k] = f32_to_bf16_bits(w);
}

// Cast of a float32 parameter vector to bf16 (round to nearest even).
__global__ void mlp_cast_kernel(const float *__restrict__ master, uint16_t *__restrict__ wb, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) wb[k] = f32_to_bf16_bits(master[k]);
}


namespace {

constexpr int kMlpThreads = 128;
constexpr size_t kParamSmem = mlp_smem_bytes(kMlpThreads);

int mlp_smem_ok() {  // per call: the attribute belongs to the current device
  int ok = 0;
  {
    ok = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kParamSmem) == cudaSuccess &&
         cudaFuncSetAttribute(mlp_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kParamSmem) == cudaSuccess;
  }
  return ok;
}

struct Scratch {
  cudaStream_t s;
  void *p = nullptr;
  Scratch(cudaStream_t st, size_t bytes) : s(st) {
    if (pool_malloc(&p, bytes, s) != cudaSuccess) p = nullptr;
  }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
};

// One training (or gradient-only) step on the batch idx[0..B) (idx null:
// samples 0..B-1).
cudaError_t enqueue_step(const uint16_t *wb, const float *x, const float *target, int64_t nsamples,
                         const int32_t *idx, int B, float *scratch, int32_t *status, float *master,
                         float *am, float *av, uint16_t *wb_out, float *grad, float *loss,
                         const AdamArgs &a, cudaStream_t s) {
  mlp_fwd_bwd_kernel<<<(B + kMlpThreads - 1) / kMlpThreads, kMlpThreads, kParamSmem, s>>>(
      wb, x, target, idx, B, nsamples, 1.0f / (float)B, scratch, status);
  mlp_grad_adam_kernel<<<(kMlpParams + 1 + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, s>>>(
      scratch, B, master, am, av, wb_out, grad, loss, a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace ga

using namespace ga;

extern "C" {

int ga_mlp_forward(const uint16_t *params_bf16, const float *x, int64_t n, float *y, void *stream) {
  if (n < 0 || (n > 0 && (!params_bf16 || !x || !y))) return GA_ERR_ARG;
  if (n == 0) return GA_OK;
  if (!mlp_smem_ok()) return GA_ERR_CUDA;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GA_ERR_CUDA;
  const int64_t want = (n + kMlpThreads - 1) / kMlpThreads;
  const int grid = (int)(want < (int64_t)nsm * 8 ? want : (int64_t)nsm * 8);
  mlp_forward_kernel<<<grid, kMlpThreads, kParamSmem, (cudaStream_t)stream>>>(params_bf16, x, n, y);
  return cudaGetLastError() == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

int ga_mlp_loss_grad(const uint16_t *params_bf16, const float *x, const float *target, int32_t n,
                     float *grad, float *loss, void *stream) {
  if (n <= 0 || !params_bf16 || !x || !target || !grad) return GA_ERR_ARG;
  if (!mlp_smem_ok()) return GA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s, sizeof(float) * (size_t)n * kScratchRow + 256);
  if (!sc.p) return GA_ERR_OOM;
  AdamArgs a{};
  a.update = 0;
  const cudaError_t e = enqueue_step(params_bf16, x, target, n, nullptr, n, (float *)sc.p, nullptr,
                                     nullptr, nullptr, nullptr, nullptr, grad, loss, a, s);
  return e == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

int ga_mlp_train(float *master, uint16_t *params_bf16, float *adam_m, float *adam_v, const float *x,
                 const float *target, int64_t nsamples, const int32_t *batch_idx, int32_t steps,
                 int32_t batch, int32_t step0, float lr, float beta1, float beta2, float eps,
                 float *losses, void *stream) {
  if (!master || !params_bf16 || !adam_m || !adam_v || !x || !target || !batch_idx) return GA_ERR_ARG;
  if (nsamples <= 0 || steps < 0 || batch <= 0 || batch > (1 << 20) || step0 < 0) return GA_ERR_ARG;
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return GA_ERR_ARG;
  if (steps == 0) return GA_OK;
  if (!mlp_smem_ok()) return GA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s, sizeof(float) * (size_t)batch * kScratchRow + 256);
  if (!sc.p) return GA_ERR_OOM;
  float *scratch = (float *)sc.p;
  Scratch st(s, 256);
  if (!st.p) return GA_ERR_OOM;
  int32_t *status = (int32_t *)st.p;
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return GA_ERR_CUDA;
  // bf16 copy of the current master weights
  mlp_cast_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(master, params_bf16, kMlpParams);

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return GA_ERR_CUDA;
  const bool graph = s != nullptr && cap == cudaStreamCaptureStatusNone && steps > 1;
  auto enqueue_all = [&]() -> cudaError_t {
    for (int k = 0; k < steps; ++k) {
      const double t = (double)step0 + k + 1;
      AdamArgs a{};
      a.lr = lr;
      a.beta1 = beta1;
      a.beta2 = beta2;
      a.eps = eps;
      a.c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, t)));
      a.c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, t)));
      a.update = 1;
      const cudaError_t e = enqueue_step(params_bf16, x, target, nsamples, batch_idx + (size_t)k * batch,
                                         batch, scratch, status, master, adam_m, adam_v, params_bf16,
                                         nullptr, losses ? losses + k : nullptr, a, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (graph) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GA_ERR_CUDA;
    const cudaError_t e1 = enqueue_all();
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return GA_ERR_CUDA;
    }
    const cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return GA_ERR_CUDA;
    const cudaError_t e4 = cudaGraphLaunch(ge, s);
    const cudaError_t e5 = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(ge);
    if (e4 != cudaSuccess || e5 != cudaSuccess) return GA_ERR_CUDA;
  } else {
    if (enqueue_all() != cudaSuccess) return GA_ERR_CUDA;
  }
  int32_t h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GA_ERR_CUDA;
  return h ? h : GA_OK;
}

int ga_mlp_cast(const float *master, uint16_t *params_bf16, void *stream) {
  if (!master || !params_bf16) return GA_ERR_ARG;
  mlp_cast_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(master, params_bf16,
                                                                                 kMlpParams);
  return cudaGetLastError() == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

}  // extern "C"
