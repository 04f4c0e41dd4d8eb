// ga_band.cuh -- pair features of the band predictor and the fused
// prediction (features -> network -> starting band w0).  Not part of the
// paper: the predictor chooses where band doubling starts, the certificate
// keeps every score exact whatever it predicts.
//
// Features of a DNA pair Q (m) / S (n), with 12-mers:
//   the k-mers of Q at positions 0, s, 2s, .. < nq = max(0, m-11),
//   s = max(1, ceil(nq / 2048)) (at most 2048 samples), go into a
//   shared-memory hash table (4096 slots, linear probing, one slot per
//   sample, so equal k-mers keep a slot each); every k-mer of S is looked up
//   and each equal sample is a hit (i, j) with diagonal d = j - i and
//   excursion e = d - clamp(d, min(0,n-m), max(0,n-m)).
//   Counts are sums over the set of hits, so they do not depend on the
//   order in which threads insert or probe.
// The 32 features (float32):
//   0..2  log2(1+m)/16, log2(1+n)/16, log2(1+|n-m|)/16
//   3     min(m,n)/max(m,n)
//   4     matched samples / samples     5  log2(1+hits)/16
//   6..13 per eighth of Q: matched samples / samples
//   14..29 hits with min(15, bitlength|e|) = b, over hits
//   30    hits with e < 0, over hits    31  1/s
#pragma once

#include "ga_dp.cuh"
#include "ga_mlp.cuh"

namespace ga {

constexpr int kFeatK = 12;
constexpr int kFeatMaxSamples = 2048;
constexpr int kFeatSlots = 4096;
constexpr int kFeatThreads = 256;
constexpr int kFeatSeg = 8;
constexpr uint32_t kFeatEmpty = 0xFFFFFFFFu;

struct BandFeatParams {
  const uint32_t *packed_q;  // flat 2-bit codes
  const uint32_t *packed_t;
  const int64_t *q_off;
  const int64_t *t_off;
  const uint8_t *qbad;       // per sequence: nonzero = invalid
  const uint8_t *tbad;
  int64_t npairs;
  float *features;           // [npairs][32] or nullptr
  // prediction (fused), when wb != nullptr
  const uint16_t *wb;        // bf16 parameters
  float margin;
  float *y;                  // nullable
  int32_t *w0;
  int32_t *status;
};

// 12 residues starting at flat position pos, first residue in the low bits
// (reads words pos/16 and pos/16 + 1; the packed buffer holds total/16 + 2
// words, so both exist for pos + 12 <= total).
__device__ __forceinline__ uint32_t kmer12(const uint32_t *base, int64_t pos) {
  const int64_t w = pos >> 4;
  const uint64_t v = (uint64_t)__ldg(base + w) | ((uint64_t)__ldg(base + w + 1) << 32);
  return (uint32_t)(v >> (2 * (int)(pos & 15))) & 0xFFFFFFu;
}

__device__ __forceinline__ int feat_slot(uint32_t key) {
  return (int)((key * 2654435761u) >> 20);  // top 12 bits
}

__device__ __forceinline__ float feat_log2(int64_t v) {  // log2(v) / 16, v >= 1
  return log2f((float)v) * 0.0625f;
}

__device__ __forceinline__ float feat_ratio(uint32_t a, uint32_t b) {
  return b ? __fdiv_rn((float)a, (float)b) : 0.f;
}

// Starting band from the network output: w0 = ceil(2^(y + margin)) - 1,
// the exponent clamped to [0, 30], w0 clamped to [0, min(m, n)] (a band of
// half-width min(m, n) already covers the matrix).
__device__ __forceinline__ int band_w0_from_y(float y, float margin, int m, int n) {
  float e = y + margin;
  e = fminf(fmaxf(e, 0.f), 30.f);
  const float wf = ceilf(exp2f(e)) - 1.f;
  int w = (int)wf;
  const int cap = m < n ? m : n;
  return w < 0 ? 0 : (w > cap ? cap : w);
}

// Dynamic shared memory: hash keys, sample positions, (PREDICT) the
// parameters as float, hit flags.
__host__ __device__ constexpr size_t feat_smem_bytes(bool predict) {
  return sizeof(uint32_t) * kFeatSlots + sizeof(int32_t) * kFeatSlots +
         (predict ? sizeof(float) * kMlpParamsPadded : 0) + kFeatSlots;
}

template <bool PREDICT>
__global__ void __launch_bounds__(kFeatThreads) band_features_kernel(const __grid_constant__ BandFeatParams p) {
  extern __shared__ __align__(16) unsigned char feat_smem[];
  uint32_t *keys = reinterpret_cast<uint32_t *>(feat_smem);
  int32_t *spos = reinterpret_cast<int32_t *>(keys + kFeatSlots);
  float *wsm = reinterpret_cast<float *>(spos + kFeatSlots);  // PREDICT: the parameters
  uint8_t *hitf = reinterpret_cast<uint8_t *>(wsm + (PREDICT ? kMlpParamsPadded : 0));
  __shared__ uint32_t cnt_hits, cnt_neg, cnt_matched;
  __shared__ uint32_t bins[16], seg_all[kFeatSeg], seg_hit[kFeatSeg];
  __shared__ float f[32];
  __shared__ float h1s[kMlpH], h2s[kMlpH];
  const int tid = threadIdx.x;
  if constexpr (PREDICT) {
    stage_params(p.wb, wsm);  // made visible by the first barrier below
  }

  for (int64_t pid = blockIdx.x; pid < p.npairs; pid += gridDim.x) {
    const int64_t qs = p.q_off[pid], ts = p.t_off[pid];
    const int m = (int)(p.q_off[pid + 1] - qs), n = (int)(p.t_off[pid + 1] - ts);
    const bool bad = (p.qbad && p.qbad[pid]) || (p.tbad && p.tbad[pid]);
    for (int k = tid; k < kFeatSlots; k += kFeatThreads) {
      keys[k] = kFeatEmpty;
      hitf[k] = 0;
    }
    if (tid < 16) bins[tid] = 0;
    if (tid < kFeatSeg) {
      seg_all[tid] = 0;
      seg_hit[tid] = 0;
    }
    if (tid == 0) {
      cnt_hits = 0;
      cnt_neg = 0;
      cnt_matched = 0;
    }
    __syncthreads();
    const int nq = m - kFeatK + 1 > 0 ? m - kFeatK + 1 : 0;
    const int stride = nq > 0 ? (nq + kFeatMaxSamples - 1) / kFeatMaxSamples : 1;
    const int ns = nq > 0 ? (nq + stride - 1) / stride : 0;
    const int nsk = n - kFeatK + 1 > 0 ? n - kFeatK + 1 : 0;
    if (!bad) {
      // insert the samples of Q (ns <= 2048 < 4096 slots: the table never fills)
      for (int k = tid; k < ns; k += kFeatThreads) {
        const int i = k * stride;
        const uint32_t key = kmer12(p.packed_q, qs + i);
        int slot = feat_slot(key);
        for (int probe = 0; probe < kFeatSlots; ++probe) {
          if (atomicCAS(&keys[slot], kFeatEmpty, key) == kFeatEmpty) {
            spos[slot] = i;
            break;
          }
          slot = (slot + 1) & (kFeatSlots - 1);
        }
        atomicAdd(&seg_all[(int)(((int64_t)kFeatSeg * i) / nq)], 1u);
      }
      __syncthreads();
      // look up every k-mer of S
      const int dlo = n - m < 0 ? n - m : 0, dhi = n - m > 0 ? n - m : 0;
      for (int j = tid; j < nsk; j += kFeatThreads) {
        const uint32_t key = kmer12(p.packed_t, ts + j);
        int slot = feat_slot(key);
        for (int probe = 0; probe < kFeatSlots; ++probe) {
          const uint32_t k2 = keys[slot];
          if (k2 == kFeatEmpty) break;
          if (k2 == key) {
            const int d = j - spos[slot];
            const int c = d < dlo ? dlo : (d > dhi ? dhi : d);
            const int e = d - c;
            const uint32_t a = (uint32_t)(e < 0 ? -e : e);
            const int b = 32 - __clz(a);
            atomicAdd(&bins[b < 15 ? b : 15], 1u);
            atomicAdd(&cnt_hits, 1u);
            if (e < 0) atomicAdd(&cnt_neg, 1u);
            hitf[slot] = 1;
          }
          slot = (slot + 1) & (kFeatSlots - 1);
        }
      }
      __syncthreads();
      for (int k = tid; k < kFeatSlots; k += kFeatThreads) {
        if (keys[k] != kFeatEmpty && hitf[k]) {
          atomicAdd(&seg_hit[(int)(((int64_t)kFeatSeg * spos[k]) / nq)], 1u);
          atomicAdd(&cnt_matched, 1u);
        }
      }
    }
    __syncthreads();
    if (tid < 32) {
      float v = 0.f;
      const int dn = n - m < 0 ? m - n : n - m;
      const uint32_t H = cnt_hits;
      if (tid == 0) v = feat_log2(1 + (int64_t)m);
      else if (tid == 1) v = feat_log2(1 + (int64_t)n);
      else if (tid == 2) v = feat_log2(1 + (int64_t)dn);
      else if (tid == 3) v = feat_ratio((uint32_t)(m < n ? m : n), (uint32_t)(m < n ? n : m));
      else if (tid == 4) v = feat_ratio(cnt_matched, (uint32_t)ns);
      else if (tid == 5) v = feat_log2(1 + (int64_t)H);
      else if (tid < 14) v = feat_ratio(seg_hit[tid - 6], seg_all[tid - 6]);
      else if (tid < 30) v = feat_ratio(bins[tid - 14], H);
      else if (tid == 30) v = feat_ratio(cnt_neg, H);
      else v = __fdiv_rn(1.f, (float)stride);
      f[tid] = v;
      if (p.features) p.features[pid * 32 + tid] = v;
    }
    if constexpr (PREDICT) {
      __syncthreads();
      // the network: thread o computes unit o with the same per-unit
      // arithmetic as the thread-per-sample kernels (same float32 result)
      if (tid < kMlpH) h1s[tid] = unit1(wsm, tid, f, 1);  // pre-activation
      __syncthreads();
      if (tid < kMlpH) h2s[tid] = fmaxf(unit2(wsm, tid, h1s, 1), 0.f);
      __syncthreads();
      if (tid == 0) {
        const float y = output(wsm, h2s, 1);
        if (p.y) p.y[pid] = y;
        p.w0[pid] = bad ? 0 : band_w0_from_y(y, p.margin, m, n);
        if (bad) set_status(p.status, GA_ERR_RESIDUE);
      }
    } else {
      if (tid == 0 && bad) set_status(p.status, GA_ERR_RESIDUE);
    }
    __syncthreads();  // the tables are reset for the next pair
  }
}

}  // namespace ga
