// ga_prot.cuh -- inter-sequence database search for alphabets of more than
// four symbols (protein), local mode: one query against many targets.
//
// The query runs along the columns and its scoring profile
// P[c][x] = sigma(query residue x, target residue c) lives in shared memory
// as int8 (Sec. 3.1, "scoring profile"), one copy per warp for the stage of
// columns it is working on (rebuilt, one 32-bit word per lane and row, from a
// transposed sigma table whenever the warp's query or stage changes);
// targets run along the rows.  As in the DNA
// inter-sequence kernel, a group of 16 lanes computes one wavefront with K
// columns per lane, and every lane carries two targets in the two int16
// halves of each register (int16x2).  For each row a lane loads the K
// profile bytes of its columns for the row residue of each half (16-byte
// shared loads) and one byte permute per column builds the packed pair of
// substitution scores.  A warp takes 4 targets of one query per task
// (targets sorted longest first, tasks query-major so that a warp keeps its
// profile for many tasks).  Queries longer than 16K columns run in stages
// of 16K columns; the right edge of a stage (packed H and outgoing F per
// row) goes to a per-group global buffer, batched through shared memory,
// that lane 0 of the next stage reads.
//
// Padding: rows past a target's end use the all-zero profile row and
// columns past the query's end have score 0; in local mode such cells
// never exceed the largest real cell, so the running maximum is exact.
// A target whose running maximum reaches 32767 - sigma_max is queued for
// an exact int32 rerun.
#pragma once

#include "ga_dp.cuh"
#include "ga_prep.cuh"

namespace ga {

constexpr int kKpG = 16;
constexpr int kKpWarps = 4;
constexpr int kKpMaxA = 31;

struct KPParams {
  const uint8_t *q_codes;
  const int64_t *q_off;
  const uint8_t *t_codes;
  const int64_t *t_off;
  const int32_t *queries;   // query ids of this launch
  int32_t nqb;
  const int32_t *t_sorted;  // valid targets, longest first
  int32_t ntv;
  int64_t nt;               // row length of `scores`
  int32_t *task_counter;
  int32_t A, alpha, beta, sigma_max_pos;
  int8_t sigma[32 * 32];    // sigma(query code, target code), A x A
  int32_t *scores;          // [nq][nt]
  int32_t *rerun_list;      // pair ids k * nt + l, rerun_cap entries
  int32_t *rerun_count;     // may exceed rerun_cap: the caller reports an error
  int32_t rerun_cap;
  int2 *bnd;                // per group slot: bnd_stride entries
  int64_t bnd_stride;
  int32_t prof_bytes;       // per warp: (A + 1) * 16K
};

// Profile layout: row c holds the stage's 16K columns.  With K = 8 or 24
// (8-byte loads) DP lane t reads its K columns at byte t*K; with K = 16 or
// 32 (16-byte loads) the row is chunk-major: 16-column chunk q of lane t
// sits at byte q*256 + t*16, so that the 8 lanes of a shared-memory phase
// read 8 different 16-byte bank groups with compile-time offsets (rows are
// multiples of 128 bytes, so the row never changes the bank).
template <int K>
__device__ __forceinline__ int prof_lane_offset(int t) {
  return (K % 16) == 0 ? t * 16 : t * K;
}
// Byte offset in a row of the K/2 columns L*K/2 .. written by lane L of the
// rebuild (they belong to DP lane L*K/2 / K).
template <int K>
__device__ __forceinline__ int prof_offset(int L) {
  constexpr int CPL = K / 2;
  const int t = L * CPL / K, c0 = L * CPL - t * K;
  if constexpr ((K % 16) == 0) return (c0 / 16) * 256 + t * 16 + (c0 % 16);
  else return L * CPL;
}

// Resident blocks per SM requested from ptxas: what shared memory allows for
// BLOSUM-sized alphabets (24 symbols + pad: (A+1) x 16K bytes of profile per
// warp plus 11.5 KB of static rings per block).
template <int K>
struct KPMinBlocks {
  static constexpr int value = K <= 8 ? 8 : K <= 16 ? 6 : K <= 24 ? 4 : 3;
};

template <int K>
__global__ void __launch_bounds__(32 * kKpWarps, KPMinBlocks<K>::value) kp_kernel(const __grid_constant__ KPParams p) {
  using Cell = CellS16x2;
  using T = uint32_t;
  constexpr int G = kKpG, W = G * K, kRing = 4 * G;
  static_assert(K % 8 == 0, "profile loads are 8 columns wide");
  extern __shared__ __align__(16) uint8_t kp_smem[];
  // sigma transposed: sigT_s[c * 32 + x] = sigma(query code x, target code c);
  // rows c >= A and columns x >= A are 0 (x = 31 is the pad column)
  __shared__ __align__(16) uint8_t sigT_s[32 * 32];
  __shared__ uint32_t ring_s[kKpWarps][2][5 * G];  // row codes of both halves, mirrored ring
  __shared__ uint2 in_ring_s[kKpWarps][2][64];
  __shared__ uint2 out_ring_s[kKpWarps][2][64];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / G, t = lane % G;
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
    const int c = i >> 5, x = i & 31;
    sigT_s[i] = (uint8_t)((c < p.A && x < p.A) ? p.sigma[x * p.A + c] : 0);
  }
  __syncthreads();
  uint8_t *prof = kp_smem + (size_t)warp * (size_t)p.prof_bytes;
  uint32_t *ring = ring_s[warp][g];
  uint2 *in_ring = in_ring_s[warp][g];
  uint2 *out_ring = out_ring_s[warp][g];
  int2 *bnd = p.bnd + (size_t)((blockIdx.x * kKpWarps + warp) * 2 + g) * (size_t)p.bnd_stride;
  const int A = p.A, alpha = p.alpha, beta = p.beta;
  const T NB = Cell::splat(-beta), NAc = Cell::splat(-alpha);
  const int ngroups = (p.ntv + 3) / 4;
  const int64_t ntasks = (int64_t)p.nqb * ngroups;
  int cur_q = -1, cur_stage = -1;  // query and stage of the profile in `prof`

  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if ((int64_t)task >= ntasks) break;
    const int k = p.queries[task / ngroups];
    const int tg = task % ngroups;
    const int64_t qs = p.q_off[k];
    const int m = (int)(p.q_off[k + 1] - qs);
    // the two targets of this group (halves 0 / 1)
    int tid[2], len[2];
    int64_t tstart[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int slot = tg * 4 + g * 2 + h;
      tid[h] = slot < p.ntv ? p.t_sorted[slot] : -1;
      tstart[h] = tid[h] >= 0 ? p.t_off[tid[h]] : 0;
      len[h] = tid[h] >= 0 ? (int)(p.t_off[tid[h] + 1] - tstart[h]) : 0;
    }
    const int Rtask = __reduce_max_sync(0xffffffffu, (unsigned)::max(len[0], len[1]));
    const int nstage = (m + W - 1) / W;
    T best = Cell::splat(0);

    for (int s = 0; s < nstage; ++s) {
      // ---- profile of this stage's columns (the whole warp) -------------
      // Lane L writes the K/2 columns L*K/2 .. of every profile row, one
      // row at a time, from the transposed sigma table (pad columns and the
      // pad row A are 0).
      if (k != cur_q || s != cur_stage) {
        __syncwarp();
        constexpr int CPL = K / 2;
        uint32_t qx4[CPL / 4];  // 4 codes per word
#pragma unroll
        for (int u = 0; u < CPL / 4; ++u) {
          uint32_t v = 0;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int col = s * W + lane * CPL + 4 * u + i;
            v |= (uint32_t)(col < m ? p.q_codes[qs + col] : 31) << (8 * i);
          }
          qx4[u] = v;
        }
        const int pofs = prof_offset<K>(lane);
        for (int c = 0; c <= A; ++c) {
          const uint8_t *row = sigT_s + c * 32;
          uint32_t w[CPL / 4];
#pragma unroll
          for (int u = 0; u < CPL / 4; ++u)
            w[u] = (uint32_t)row[qx4[u] & 0xffu] | ((uint32_t)row[(qx4[u] >> 8) & 0xffu] << 8) |
                   ((uint32_t)row[(qx4[u] >> 16) & 0xffu] << 16) | ((uint32_t)row[qx4[u] >> 24] << 24);
          uint8_t *dst = prof + (size_t)c * W + pofs;
          if constexpr (CPL == 16) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
          } else if constexpr (CPL == 8) {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(w[0], w[1]);
          } else {
#pragma unroll
            for (int u = 0; u < CPL / 4; ++u) reinterpret_cast<uint32_t *>(dst)[u] = w[u];
          }
        }
        cur_q = k;
        cur_stage = s;
        __syncwarp();
      }
      // ---- row codes of both halves, refilled G rows ahead ---------------
      auto fill_batch = [&](int b) {
        const int r = b * G + 1 + t;
        const uint32_t c0 = r <= len[0] ? p.t_codes[tstart[0] + r - 1] : (uint32_t)A;
        const uint32_t c1 = r <= len[1] ? p.t_codes[tstart[1] + r - 1] : (uint32_t)A;
        const int sl = r & (kRing - 1);
        const uint32_t v = c0 | (c1 << 16);
        ring[sl] = v;
        if (sl < G) ring[sl + kRing] = v;
      };
      // left edge of the stage, batched (rows 16b+1 .. 16b+16)
      auto load_edge = [&](int b) {
        if (s > 0) {
          const int r = b * G + 1 + t;
          if (r <= Rtask) {
            const int2 v = bnd[r];
            in_ring[(r - 1) & 63] = make_uint2((uint32_t)v.x, (uint32_t)v.y);
          }
        }
      };
      __syncwarp();
      fill_batch(0);
      fill_batch(1);
      load_edge(0);
      __syncwarp();

      T H[K], E[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        H[j] = Cell::splat(0);
        E[j] = NAc;  // E(1, j) = H(0, j) - alpha
      }
      auto left = [&](int r, T &hl, T &fl) {  // lane 0: (H(r, 16Ks), F(r, 16Ks+1))
        if (s == 0) {
          hl = Cell::splat(0);
          fl = NAc;
        } else {
          const uint2 v = in_ring[(r - 1) & 63];
          hl = v.x;
          fl = v.y;
        }
      };
      T Hdiag = Cell::splat(0), Hleft = Cell::splat(0), Fin = Cell::splat(CellInfo<Cell>::kNeg);
      if (t == 0) left(1, Hleft, Fin);

      const int nit = Rtask + G - 1;
      for (int it = 0; it < nit; ++it) {
        if ((it % G) == 0) {
          __syncwarp();
          fill_batch(it / G + 2);
          load_edge(it / G + 1);
          if (it >= 2 * G) {  // flush lane 15's rows it-31 .. it-16
            const int r = it - 2 * G + 1 + t;
            const uint2 v = out_ring[(r - 1) & 63];
            bnd[r] = make_int2((int)v.x, (int)v.y);
          }
          __syncwarp();
        }
        const int r = it - t + 1;
        T Hout = H[K - 1], Fout = Cell::splat(CellInfo<Cell>::kNeg);
        if ((unsigned)(r - 1) < (unsigned)Rtask) {
          const uint32_t rc = ring[r & (kRing - 1)];
          const uint8_t *b0 = prof + (size_t)(rc & 0xffffu) * W + prof_lane_offset<K>(t);
          const uint8_t *b1 = prof + (size_t)(rc >> 16) * W + prof_lane_offset<K>(t);
          uint32_t w0[K / 4], w1[K / 4];
          if constexpr ((K % 16) == 0) {  // chunk-major rows, 16-byte loads
#pragma unroll
            for (int q = 0; q < K / 16; ++q) {
              const uint4 a = *reinterpret_cast<const uint4 *>(b0 + q * 256);
              const uint4 b = *reinterpret_cast<const uint4 *>(b1 + q * 256);
              w0[4 * q] = a.x; w0[4 * q + 1] = a.y; w0[4 * q + 2] = a.z; w0[4 * q + 3] = a.w;
              w1[4 * q] = b.x; w1[4 * q + 1] = b.y; w1[4 * q + 2] = b.z; w1[4 * q + 3] = b.w;
            }
          } else {  // 8-byte boundaries (K = 8, 24)
#pragma unroll
            for (int q = 0; q < K / 8; ++q) {
              const uint2 a = reinterpret_cast<const uint2 *>(b0)[q];
              const uint2 b = reinterpret_cast<const uint2 *>(b1)[q];
              w0[2 * q] = a.x; w0[2 * q + 1] = a.y;
              w1[2 * q] = b.x; w1[2 * q + 1] = b.y;
            }
          }
          Fout = dp_row<Cell, kModeLocal, K>(
              H, E, Hdiag, Fin, NB, best,
              [&](int j) -> T { return (T)prmt(w0[j >> 2], w1[j >> 2], sext_sel<Cell>(j & 3)); },
              [&](int) -> T { return NAc; });
          Hout = H[K - 1];
          if (t == G - 1) out_ring[(r - 1) & 63] = make_uint2(Hout, Fout);
        }
        Hdiag = Hleft;
        Hleft = __shfl_up_sync(0xffffffffu, Hout, 1, G);
        Fin = __shfl_up_sync(0xffffffffu, Fout, 1, G);
        if (t == 0) {
          if (it + 2 <= Rtask) left(it + 2, Hleft, Fin);
          else {
            Hleft = Cell::splat(0);
            Fin = NAc;
          }
        }
      }
      __syncwarp();
      if (s + 1 < nstage) {  // flush the remaining rows of the edge
        const int first = (nit - 1 >= 2 * G) ? ((nit - 1) / G) * G - 2 * G + 1 + G : 1;
        for (int r = first + t; r <= Rtask; r += G) {
          const uint2 v = out_ring[(r - 1) & 63];
          bnd[r] = make_int2((int)v.x, (int)v.y);
        }
      }
      __syncwarp();
    }

    // ---- scores ----------------------------------------------------------
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = group_max<G>(cell_get<Cell>(best, h));
      if (tid[h] >= 0 && t == 0) {
        const int64_t pid = (int64_t)k * p.nt + tid[h];
        if (v >= 32767 - p.sigma_max_pos) {
          const int sl = atomicAdd(p.rerun_count, 1);
          if (sl < p.rerun_cap) p.rerun_list[sl] = (int32_t)pid;
        } else {
          p.scores[pid] = v;
        }
      }
    }
    __syncwarp();
  }
}

// Sort keys of the targets: longest first (the row buckets of the plan
// kernel), invalid targets left out; the longest valid target length goes
// to *max_len.
__global__ void kp_target_keys_kernel(const int64_t *t_off, int64_t nt, const uint8_t *tbad, uint32_t *keys,
                                      int32_t *max_len) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int L = 0;
  if (i < nt) {
    uint32_t key = 0xffffffffu;
    if (!tbad[i]) {
      const int64_t n = t_off[i + 1] - t_off[i];
      const int64_t rb = n < 1536 ? n : (1536 + ((n - 1536) >> 6) < kRBuckets - 1 ? 1536 + ((n - 1536) >> 6)
                                                                                  : kRBuckets - 1);
      key = (uint32_t)(kRBuckets - 1 - rb);
      L = (int)(n < (1 << 30) ? n : (1 << 30));
    }
    keys[i] = key;
  }
  L = (int)__reduce_max_sync(0xffffffffu, (unsigned)L);
  if ((threadIdx.x & 31) == 0 && L > 0) atomicMax(max_len, L);
}

// Scores of pairs with an invalid query or target.
__global__ void kp_invalid_kernel(const uint8_t *qbad, int64_t nq, const uint8_t *tbad, int64_t nt,
                                  int32_t *scores, int32_t *status) {
  const int64_t total = nq * nt;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / nt, l = i - k * nt;
    if (qbad[k] || tbad[l]) {
      scores[i] = INT32_MIN;
      set_status(status, (qbad[k] == 2 || tbad[l] == 2) ? GA_ERR_ARG : GA_ERR_RESIDUE);
    }
  }
}

// Rows / columns / offsets of the pairs to rerun (for the host loop).
__global__ void kp_rerun_info_kernel(const int32_t *list, int32_t n, int64_t nt, const int64_t *q_off,
                                     const int64_t *t_off, int64_t *out /* [n][4]: qs, m, ts, n */) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t pid = list[i], k = pid / nt, l = pid - k * nt;
  out[4 * i] = q_off[k];
  out[4 * i + 1] = q_off[k + 1] - q_off[k];
  out[4 * i + 2] = t_off[l];
  out[4 * i + 3] = t_off[l + 1] - t_off[l];
}

}  // namespace ga
