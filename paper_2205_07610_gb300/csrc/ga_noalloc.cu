// ga_noalloc.cu -- ga_align_long_noalloc: the long-pair kernel with its
// scratch memory in a fixed, file-scope device array instead of memory
// allocated per call.
//
// Who needs it: a caller that cannot allocate device memory at the moment it
// aligns -- for example a process whose memory has been handed in full to a
// pooling allocator (so cudaMalloc fails), or a latency-critical loop that
// cannot afford the implicit device synchronisation and unbounded latency of
// cudaMalloc/cudaFree.  This entry point calls neither cudaMalloc, cudaFree,
// cudaMallocAsync nor any other allocating routine.
//
// The array (about 2 MiB) is loaded with the library onto every GPU that
// uses it and stays there until the process exits.  Every call shares it:
// calls whose work overlaps on the GPU (different streams, or different host
// threads without ordering) race on it and must be serialised by the caller.
// The array keeps the last call's contents; the preparation kernel rewrites
// every field that must start fresh (task counter, status, offsets) before
// the DP kernel reads it.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "ga_launch.h"

namespace ga {
namespace {

// Longest sequence accepted (rows of the DP after orientation).
constexpr int64_t kNoAllocMaxLen = GA_NOALLOC_MAX_LEN;
constexpr int64_t kNoAllocBndStride = kNoAllocMaxLen + 128;  // kb_kernel reads up to R + 94
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocCtl {
  int64_t q_off[2];
  int64_t t_off[2];
  int4 info;
  int32_t sorted;
  int32_t range[2];
  int32_t counter;
  int32_t status;
  int32_t pad[3];
};

constexpr size_t kCtlBytes = (sizeof(NoAllocCtl) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCtlBytes + (size_t)kKbWarps * kNoAllocBndStride * sizeof(int2);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array, looked up once per device (host code must not
// use the symbol itself: on the host it is only a stand-in).
void *g_scratch_ptr[kNoAllocMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GA_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GA_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GA_OK;
}

// One warp: validate the residues, orient the pair, fill the control block
// and write trivial or invalid results directly.
__global__ void noalloc_prep_kernel(NoAllocCtl *ctl, const uint8_t *q, int64_t m, const uint8_t *t,
                                    int64_t n, int A, int mode, int alpha, int beta,
                                    int32_t *score) {
  const int lane = threadIdx.x & 31;
  unsigned mx = 0;
  for (int64_t i = lane; i < m; i += 32) mx = max(mx, (unsigned)q[i]);
  for (int64_t i = lane; i < n; i += 32) mx = max(mx, (unsigned)t[i]);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane != 0) return;
  ctl->q_off[0] = 0;
  ctl->q_off[1] = m;
  ctl->t_off[0] = 0;
  ctl->t_off[1] = n;
  ctl->sorted = 0;
  ctl->counter = 0;
  ctl->status = GA_OK;
  ctl->range[0] = 0;
  ctl->range[1] = 0;
  if ((m > 0 || n > 0) && mx >= (unsigned)A) {
    ctl->status = GA_ERR_RESIDUE;
    *score = INT32_MIN;
    return;
  }
  if (m == 0 || n == 0) {
    const int64_t len = m + n;
    *score = (mode == GA_GLOBAL && len > 0) ? -(int)(alpha + beta * (len - 1)) : 0;
    return;
  }
  const int64_t R = m >= n ? m : n, C = m >= n ? n : m;
  ctl->info = make_int4((int)R, (int)C, m < n ? 1 : 0, (int)kClassLong);
  ctl->range[1] = 1;
}

}  // namespace
}  // namespace ga

using namespace ga;

extern "C" int ga_align_long_noalloc(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                                     const ga_scoring *scoring, int32_t mode, int32_t *score,
                                     void *stream) {
  if (m < 0 || n < 0 || !score || (m > 0 && !q) || (n > 0 && !t)) return GA_ERR_ARG;
  if (mode < 0 || mode > 2) return GA_ERR_ARG;
  if (m > kNoAllocMaxLen || n > kNoAllocMaxLen) return GA_ERR_ARG;
  if (!scoring) return GA_ERR_ARG;
  if (scoring->alphabet_size < 1 || scoring->alphabet_size > 31 || !scoring->matrix)
    return GA_ERR_ALPHABET;
  if (scoring->gap_open <= 0 || scoring->gap_extend <= 0 || scoring->gap_extend > scoring->gap_open ||
      scoring->gap_open > 4096)
    return GA_ERR_ARG;
  const int A = scoring->alphabet_size;
  int64_t bound = 0;
  int smax = 0;
  for (int i = 0; i < A * A; ++i) {
    if (scoring->matrix[i] < -127) return GA_ERR_ALPHABET;
    smax = std::max(smax, std::abs((int)scoring->matrix[i]));
  }
  bound = (int64_t)smax * std::min(m, n) + 3 * (int64_t)scoring->gap_open +
          (int64_t)scoring->gap_extend * (m + n);
  if (bound >= (1ll << 30)) return GA_ERR_RANGE;

  void *base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  NoAllocCtl *ctl = (NoAllocCtl *)base;
  int2 *bnd = (int2 *)((unsigned char *)base + kCtlBytes);
  cudaStream_t s = (cudaStream_t)stream;

  noalloc_prep_kernel<<<1, 32, 0, s>>>(ctl, q, m, t, n, A, mode, scoring->gap_open,
                                       scoring->gap_extend, score);
  if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;

  KBParams kb{};
  kb.q_codes = q;
  kb.t_codes = t;
  kb.q_off = ctl->q_off;
  kb.t_off = ctl->t_off;
  kb.info = &ctl->info;
  kb.sorted = &ctl->sorted;
  kb.range = ctl->range;
  kb.task_counter = &ctl->counter;
  for (int i = 0; i < A * A; ++i) kb.sigma[i] = scoring->matrix[i];
  kb.A = A;
  kb.alpha = scoring->gap_open;
  kb.beta = scoring->gap_extend;
  kb.scores = score;
  kb.bnd = bnd;
  kb.bnd_stride = kNoAllocBndStride;
  kb.nt = 0;
  kb.q0 = 0;
  const size_t smem = (size_t)kKbWarps * (size_t)(A + 1) * (32 * kKbK);
  cudaError_t e = mode == GA_LOCAL ? launch_kb_local_prof(kb, 1, smem, s)
                : mode == GA_GLOBAL ? launch_kb_global_prof(kb, 1, smem, s)
                                    : launch_kb_semi_prof(kb, 1, smem, s);
  return e == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}
