// ga_prep.cuh -- encode / validate / classify / length-sort kernels.
//
// a1: residue codes are checked against the alphabet and, for alphabets of
//     <= 4 symbols, packed 2 bits per residue (16 per 32-bit word; sequence
//     k starts at word off[k]/16 + k, which needs no prefix sum because a
//     sequence of length L never needs more than floor(L/16) + 1 words
//     beyond the word of its first residue).
// a2: every pair is classified (packed int16x2 / int32 inter-sequence
//     kernel, long kernel, or done: empty or invalid), oriented (rows = the
//     longer sequence), binned by its column count and keyed by its row
//     count; a counting sort groups pairs by (class, bin) with long rows
//     first, so a task's pairs have similar lengths and the longest work
//     starts first.
#pragma once

#include "ga_common.cuh"

namespace ga {

constexpr int kBins = 18;  // >= the inter-sequence tiles (17)
constexpr int kRBuckets = 2048;  // exact rows below 1536, then 64-row steps
constexpr int kClassesSorted = 3;  // inter16, inter32, long
constexpr int kNumKeys = kClassesSorted * kBins * kRBuckets;

// Column-count limits of the inter-sequence bins (W = G*K per bin).
struct BinTable {
  int n16;            // bins of the int16x2 kernel for this mode
  int w16[kBins];
  int n32;
  int w32[kBins];
};

struct PlanParams {
  const int64_t *q_off;
  const int64_t *t_off;
  int64_t npairs;             // pairs (batch) or combinations of this chunk (cross)
  int64_t nt;                 // cross: targets per query (0: batch, pair p = (p, p))
  int64_t q0;                 // cross: first query of this chunk
  const uint8_t *qbad;        // per query sequence: 0 ok, 1 residue, 2 offsets
  const uint8_t *tbad;
  int32_t A;
  int32_t mode;
  int32_t alpha, beta;
  int32_t sigma_max, sigma_min;
  int32_t dna;                // alphabet packed 2-bit (<= 4 symbols)
  BinTable bins;
  int32_t *scores;
  uint32_t *keys;
  int4 *info;
  int32_t *status;
  unsigned long long *cells;  // sum m*n over valid pairs
  int32_t *rmax_long;         // max rows over long-class pairs
};

// 2-bit codes of the 4 bytes of x (low 2 bits of each byte) in 8 bits.
__device__ __forceinline__ uint32_t pack4(uint32_t x) {
  uint32_t y = x & 0x03030303u;
  y = (y | (y >> 6)) & 0x000f000fu;
  return (y | (y >> 12)) & 0xffu;
}

// Flat 2-bit packing of the whole code buffer (residue x -> word x/16),
// one thread per word with a 16-byte load; any code >= A anywhere raises
// *invalid (per-sequence validation then runs its slow path).
__device__ __forceinline__ void flat_pack_body(const uint8_t *codes, int64_t start, int64_t total, int A,
                                               uint32_t *packed, int32_t *invalid) {
  // words start/16 .. (total+15)/16 - 1: the residues [start, total) and the
  // bytes before `start` in its word (which exist: they are codes of the
  // same buffer)
  const int64_t nwords = (total + 15) / 16;
  const int64_t w_first = start / 16;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(codes) & 15u) == 0;
  const uint32_t A4 = (uint32_t)A * 0x01010101u;
  bool bad = false;
  for (int64_t w = w_first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = w * 16;
    uint32_t x[4];
    if (aligned16 && s0 + 16 <= total) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(codes + s0));
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (s0 + 4 * i + j < total) acc |= (uint32_t)codes[s0 + 4 * i + j] << (8 * j);
        x[i] = acc;  // bytes past the end are 0, a valid code
      }
    }
    uint32_t word = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      bad |= __vcmpgeu4(x[i], A4) != 0u;
      word |= pack4(x[i]) << (8 * i);
    }
    if (packed) packed[w] = word;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(invalid, 1);
}

__global__ void flat_pack_kernel(const uint8_t *codes, int64_t start, int64_t total, int A,
                                 uint32_t *packed, int32_t *invalid) {
  flat_pack_body(codes, start, total, A, packed, invalid);
}

// Flat 5-bit packing of the code buffer for alphabets of up to 32 symbols
// (protein): residue x of the buffer sits in word x / 6 at bits 5 (x % 6)
// .. 5 (x % 6) + 4, six residues per word.  One thread per 8 words (48
// residues: three 16-byte loads when the chunk is aligned and complete, two
// 16-byte stores); any code >= A raises *invalid as in the 2-bit packing.
__global__ void flat_pack5_kernel(const uint8_t *codes, int64_t start, int64_t total, int A,
                                  uint32_t *packed5, int32_t *invalid) {
  const int64_t nwords = (total + 5) / 6;
  const int64_t w_first = start / 6 / 8 * 8;  // chunks of 8 words from an 8-word boundary
  const bool aligned16 = (reinterpret_cast<uintptr_t>(codes) & 15u) == 0;
  bool bad = false;
  for (int64_t w0 = w_first + 8 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); w0 < nwords;
       w0 += 8 * (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = w0 * 6;  // 48 residues, s0 a multiple of 48 (16-byte aligned offset)
    uint8_t r[48];
    if (aligned16 && s0 + 48 <= total && s0 >= start) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(codes + s0) + k);
        const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) r[16 * k + i] = (uint8_t)(x[i >> 2] >> (8 * (i & 3)));
      }
    } else {
#pragma unroll
      for (int i = 0; i < 48; ++i) r[i] = (s0 + i >= start && s0 + i < total) ? codes[s0 + i] : (uint8_t)0;
    }
    uint32_t out[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t word = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const uint32_t c = r[6 * k + i];
        bad |= c >= (uint32_t)A;
        word |= (c & 31u) << (5 * i);
      }
      out[k] = word;
    }
    if (w0 + 8 <= nwords) {
      reinterpret_cast<uint4 *>(packed5 + w0)[0] = make_uint4(out[0], out[1], out[2], out[3]);
      reinterpret_cast<uint4 *>(packed5 + w0)[1] = make_uint4(out[4], out[5], out[6], out[7]);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (w0 + k < nwords) packed5[w0 + k] = out[k];
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(invalid, 1);
}

// Batch plans: the residue range [off[0], off[nseq]) of a set is read on
// the device and clamped to the plan's capacity `cap` (residues at or
// beyond cap are never read; validation marks their sequences).
__global__ void plan_pack_kernel(const uint8_t *codes, const int64_t *off, int64_t nseq, int64_t cap, int A,
                                 uint32_t *packed, int32_t *invalid) {
  const int64_t e = off[nseq], b = off[0];
  const int64_t total = e < 0 ? 0 : (e < cap ? e : cap);
  const int64_t start = b < 0 ? 0 : (b < total ? b : total);
  flat_pack_body(codes, start, total, A, packed, invalid);
}

// Thread per sequence of a plan run: 0 ok, 1 residue code >= A, 2 offsets
// decreasing (or off[0] < 0), 3 sequence longer than max_len or ending
// beyond cap.
__global__ void plan_validate_kernel(const uint8_t *codes, const int64_t *off, int64_t nseq, int64_t cap,
                                     int64_t max_len, int A, const int32_t *invalid, uint8_t *bad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nseq) return;
  const int64_t first = off[0], last = off[nseq];
  const int64_t s = off[k], e = off[k + 1];
  uint8_t b = 0;
  if (first < 0 || s < first || e < s || e > last) {
    b = 2;
  } else if (e > cap || e - s > max_len) {
    b = 3;
  } else if (*invalid) {
    for (int64_t x = s; x < e; ++x)
      if (codes[x] >= (unsigned)A) { b = 1; break; }
  }
  bad[k] = b;
}

// Thread per sequence: 0 ok, 1 residue code >= A, 2 offsets decreasing or
// outside [start, total] (start = off[0], total = off[nseq]).  Residues are scanned only when the packing pass saw
// an invalid code somewhere.
__global__ void validate_kernel(const uint8_t *codes, const int64_t *off, int64_t nseq,
                                int64_t start, int64_t total, int A, const int32_t *invalid,
                                uint8_t *bad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nseq) return;
  const int64_t s = off[k], e = off[k + 1];
  uint8_t b = 0;
  if (s < start || e < s || e > total) {
    b = 2;
  } else if (*invalid) {
    for (int64_t x = s; x < e; ++x)
      if (codes[x] >= (unsigned)A) { b = 1; break; }
  }
  bad[k] = b;
}

__device__ __forceinline__ int global_gap(int alpha, int beta, int64_t len) {
  return len == 0 ? 0 : -(int)(alpha + beta * (len - 1));
}

// One pair (batch) or (query, target) combination (cross chunk).
__device__ __forceinline__ void plan_one(const PlanParams &p, int64_t i, unsigned long long &my_cells) {
  const int64_t qi = p.nt ? p.q0 + i / p.nt : i;
  const int64_t ti = p.nt ? i % p.nt : i;
  const int64_t m = p.q_off[qi + 1] - p.q_off[qi];
  const int64_t n = p.t_off[ti + 1] - p.t_off[ti];
  int4 inf = make_int4(0, 0, 0, (int)kClassDone);
  uint32_t key = 0xffffffffu;
  const uint8_t qb = p.qbad[qi], tb = p.tbad[ti];
  if (qb || tb || m < 0 || n < 0) {
    p.scores[i] = INT32_MIN;
    set_status(p.status, (qb == 2 || tb == 2 || m < 0 || n < 0) ? GA_ERR_ARG
                         : (qb == 3 || tb == 3)                  ? GA_ERR_RANGE
                                                                 : GA_ERR_RESIDUE);
  } else if (m == 0 || n == 0) {
    p.scores[i] = (p.mode == GA_GLOBAL) ? global_gap(p.alpha, p.beta, m + n) : 0;
  } else {
    const int64_t R = m >= n ? m : n, C = m >= n ? n : m;
    const int swap = m < n;
    const int64_t smax = p.sigma_max > 0 ? p.sigma_max : 0;
    const int64_t sabs = max(smax, (int64_t)(p.sigma_min < 0 ? -p.sigma_min : 0));
    // int32 admissibility: every reachable value stays well inside int32.
    const int64_t bound32 = sabs * C + 3 * (int64_t)p.alpha + (int64_t)p.beta * (R + C);
    if (bound32 >= (1ll << 30) || R >= (1ll << 30)) {
      p.scores[i] = INT32_MIN;
      set_status(p.status, GA_ERR_RANGE);
    } else {
      my_cells = (unsigned long long)(m * n);
      uint32_t cls = kClassLong;
      int bin = 0;
      if (p.dna) {
        // smallest int16x2 bin that fits the columns, if int16 is exact
        int b16 = -1, b32 = -1;
        for (int b = 0; b < p.bins.n16; ++b)
          if (C <= p.bins.w16[b]) { b16 = b; break; }
        for (int b = 0; b < p.bins.n32; ++b)
          if (C <= p.bins.w32[b]) { b32 = b; break; }
        bool ok16 = b16 >= 0 && p.alpha <= kInt16MaxGap && p.beta <= kInt16MaxGap;
        if (ok16) {
          const int64_t W = p.bins.w16[b16];
          const int64_t up = smax * C;
          int64_t lo;
          if (p.mode == GA_GLOBAL) lo = 2 * (int64_t)p.alpha + (int64_t)p.beta * (R + C);
          else if (p.mode == GA_SEMIGLOBAL) lo = (int64_t)p.alpha * (W - C + 2) + (int64_t)p.beta * C;
          else lo = p.alpha;
          // local: values are >= 0; an overflow of the upper bound is
          // detected at run time and the pair is redone in int32.
          if (p.mode != GA_LOCAL && up > kInt16Bound) ok16 = false;
          if (lo > kInt16Bound) ok16 = false;
        }
        if (ok16) { cls = kClassInter16; bin = b16; }
        else if (b32 >= 0) { cls = kClassInter32; bin = b32; }
      }
      if (cls == kClassLong) atomicMax(p.rmax_long, (int)R);
      inf = make_int4((int)R, (int)C, swap, (int)cls);
      const int64_t rb = R < 1536 ? R : (1536 + ((R - 1536) >> 6) < kRBuckets - 1 ? 1536 + ((R - 1536) >> 6) : kRBuckets - 1);
      key = (uint32_t)(((cls * kBins + bin) * kRBuckets) + (kRBuckets - 1 - rb));
    }
  }
  p.info[i] = inf;
  p.keys[i] = key;
}

__global__ void plan_kernel(PlanParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long my_cells = 0;
  if (i < p.npairs) plan_one(p, i, my_cells);
  // one atomic per warp for the cell count
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) my_cells += __shfl_xor_sync(0xffffffffu, my_cells, off);
  if ((threadIdx.x & 31) == 0 && my_cells) atomicAdd(p.cells, my_cells);
}

// Banded path: invalid / empty pairs are finished here, the others are
// keyed by estimated work m * (|n-m| + 2 w0 + 1), largest first.
struct BandPlanParams {
  const int64_t *q_off;
  const int64_t *t_off;
  int64_t npairs;
  const uint8_t *qbad;
  const uint8_t *tbad;
  const int32_t *w0;
  int32_t default_w0;
  int32_t alpha, beta;
  int32_t *scores;
  int32_t *w_used;
  uint32_t *keys;
  int32_t *status;
  unsigned long long *cells;
  int32_t *max_rows;
  int32_t *max_span;   // max of max(m + 1, 128) x super-stages + m, saturated
  int32_t stage_cols;  // columns of a super-stage of the packed band kernel
};

__global__ void band_plan_kernel(BandPlanParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long my_cells = 0;
  if (i < p.npairs) {
    const int64_t m = p.q_off[i + 1] - p.q_off[i], n = p.t_off[i + 1] - p.t_off[i];
    int w = p.w0 ? p.w0[i] : p.default_w0;
    if (w < 0) w = 0;
    uint32_t key = 0xffffffffu;
    if (p.qbad[i] || p.tbad[i] || m < 0 || n < 0) {
      p.scores[i] = INT32_MIN;
      if (p.w_used) p.w_used[i] = -1;
      set_status(p.status, (p.qbad[i] == 2 || p.tbad[i] == 2) ? GA_ERR_ARG : GA_ERR_RESIDUE);
    } else if (m >= (1ll << 30) || n >= (1ll << 30) ||
               2 * (int64_t)p.alpha + (int64_t)p.beta * (m + n) + 127 * (m < n ? m : n) >= (1ll << 30)) {
      p.scores[i] = INT32_MIN;
      if (p.w_used) p.w_used[i] = -1;
      set_status(p.status, GA_ERR_RANGE);
    } else if (m == 0 || n == 0) {
      p.scores[i] = global_gap(p.alpha, p.beta, m + n);
      if (p.w_used) p.w_used[i] = w;
    } else {
      my_cells = (unsigned long long)(m * n);
      atomicMax(p.max_rows, (int)m);
      {
        // bound on the packed band kernel's iteration numbers: its super-
        // stages are at most max(m + 1, 128) iterations apart
        const int64_t span = (m + 1 > 128 ? m + 1 : 128) * ((n + p.stage_cols - 1) / p.stage_cols) + m;
        atomicMax(p.max_span, (int)(span < INT32_MAX ? span : INT32_MAX));
      }
      // The band kernels take pairs from a queue in this order, so the key
      // puts the most work first (the last pairs to start are the short
      // ones): super-stages of stage_cols columns (exact up to 31), then the
      // length of a block's row window, 2w + |n - m| + 16 (four buckets per
      // octave).
      const int64_t d = n - m;
      const int64_t nst = (n + p.stage_cols - 1) / p.stage_cols;
      const int64_t L = (d < 0 ? -d : d) + 2 * (int64_t)w + 16;
      const int lg = 63 - __clzll((long long)L);
      const int lb = ::min(63, lg * 4 + (int)((L >> (lg - 2)) & 3));
      key = (uint32_t)(kRBuckets - 1 - (int)((nst < 31 ? nst : 31) * 64 + lb));
    }
    p.keys[i] = key;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) my_cells += __shfl_xor_sync(0xffffffffu, my_cells, off);
  if ((threadIdx.x & 31) == 0 && my_cells) atomicAdd(p.cells, my_cells);
}

__global__ void hist_kernel(const uint32_t *keys, int64_t n, int32_t *hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i];
  if (k != 0xffffffffu) atomicAdd(&hist[k], 1);
}

// Exclusive scan of hist -> cursor and the [start, end) range of every
// (class, bin) in ranges[2 * (class * kBins + bin)], in two launches over
// tiles of 1024 buckets: per-tile totals, then per-tile scans offset by the
// totals of the tiles before.
constexpr int kScanTile = 1024;
constexpr int kScanTiles = kNumKeys / kScanTile;
static_assert(kNumKeys % kScanTile == 0, "scan tiling");

__device__ __forceinline__ int32_t block_sum_1024(int32_t v, int32_t *sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = __reduce_add_sync(0xffffffffu, (unsigned)v);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  int32_t tot = 0;
  if (warp == 0) {
    tot = __reduce_add_sync(0xffffffffu, (unsigned)sm[lane]);
    if (lane == 0) sm[32] = tot;
  }
  __syncthreads();
  return sm[32];
}

__global__ void scan_partials_kernel(const int32_t *hist, int32_t *partials) {
  __shared__ int32_t sm[33];
  const int32_t v = hist[blockIdx.x * kScanTile + threadIdx.x];
  const int32_t tot = block_sum_1024(v, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void scan_apply_kernel(const int32_t *hist, const int32_t *partials, int32_t *cursor,
                                  int32_t *ranges) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t base_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    int32_t acc = 0;
    for (int b = lane; b < (int)blockIdx.x; b += 32) acc += partials[b];
    acc = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)acc);
    if (lane == 0) base_s = acc;
  }
  const int k = blockIdx.x * kScanTile + threadIdx.x;
  const int32_t v = hist[k];
  int32_t incl = v;  // inclusive warp scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t w = wsum[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    wsum[lane] = wi - w;  // exclusive over warps
  }
  __syncthreads();
  const int32_t excl = base_s + wsum[warp] + incl - v;
  cursor[k] = excl;
  if ((k % kRBuckets) == 0) ranges[2 * (k / kRBuckets)] = excl;
  if ((k % kRBuckets) == kRBuckets - 1) ranges[2 * (k / kRBuckets) + 1] = excl + v;
}

__global__ void scatter_kernel(const uint32_t *keys, int64_t n, int32_t *cursor, int32_t *sorted) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i];
  if (k == 0xffffffffu) return;
  const int pos = atomicAdd(&cursor[k], 1);
  sorted[pos] = (int32_t)i;
}

// Writes {0, count} so a kernel can take its range from a device counter.
__global__ void range_from_count_kernel(const int32_t *count, int32_t *range) {
  range[0] = 0;
  range[1] = *count;
}

}  // namespace ga
