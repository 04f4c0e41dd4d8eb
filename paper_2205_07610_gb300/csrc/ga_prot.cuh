// ga_prot.cuh -- inter-sequence database search for alphabets of more than
// four symbols (protein), local mode: many queries against many targets.
//
// Queries run along the columns, targets along the rows.  As in the DNA
// inter-sequence kernel a group of 16 lanes computes one wavefront with K
// columns per lane, and every register carries two alignments in its two
// int16 halves; here the halves are two queries of similar length against
// the same target, so that both halves of a row share the row residue c and
// the scoring profile (Sec. 3.1, "scoring profile") can hold the packed
// pair directly:
//
//   P[c][x] = sigma(query0[x], c) | sigma(query1[x], c) << 16   (int16x2)
//
// One profile per block, in shared memory, for the stage of 16K columns the
// block is working on: the 4 warps (8 groups) of a block take 8 targets of
// one query pair per task (targets sorted longest first, tasks
// query-pair-major), and the block rebuilds the profile from a transposed
// sigma table only when its query pair or stage changes.  A row then costs
// K/4 16-byte shared loads per lane and no per-column byte permute.
// Queries longer than 16K columns run in stages of 16K columns; lane 15
// stores the right edge of a stage (packed H and outgoing F per row) to a
// per-group global buffer, which the next stage reads back in batches of
// 16 rows through shared memory for its lane 0.
//
// Padding: rows past a target's end use the all-zero profile row and
// columns past a query's end have score 0; in local mode such cells never
// exceed the largest real cell, so the running maximum is exact.  A pair
// whose running maximum reaches 32767 - sigma_max is queued for an exact
// int32 rerun: its score entry is set to kRerunMark (no real score comes
// near it: every admitted score is below 2^30) and its id is appended to the
// rerun list while the list has room, so the caller can always find every
// flagged pair by scanning the scores when the list overflowed.
#pragma once

#include "ga_dp.cuh"
#include "ga_prep.cuh"

namespace ga {

constexpr int kKpG = 16;
constexpr int kKpWarps = 4;
constexpr int kKpGroups = 2 * kKpWarps;  // targets per block task
constexpr int kKpMaxA = 31;
constexpr int32_t kRerunMark = 0x7fffffff;

struct KPParams {
  const uint8_t *q_codes;
  const int64_t *q_off;
  const uint8_t *t_codes;
  const uint32_t *t_packed5;  // the target codes packed 5 bits each (flat_pack5_kernel)
  const int64_t *t_off;
  const int32_t *queries;   // query ids of this launch; entries 2i, 2i+1 form pair i
  int32_t nqb;
  const int32_t *t_sorted;  // valid targets, longest first
  int32_t ntv;
  int64_t nt;               // row length of `scores`
  int32_t *task_counter;
  int32_t A, alpha, beta, sigma_max_pos;
  int8_t sigma[32 * 32];    // sigma(query code, target code), A x A
  int32_t *scores;          // [nq][nt]
  int32_t *rerun_list;      // pair ids k * nt + l, rerun_cap entries
  int32_t *rerun_count;     // may exceed rerun_cap: the caller then scans for kRerunMark
  int32_t rerun_cap;
  int2 *bnd;                // per group slot: bnd_stride entries
  int64_t bnd_stride;
};

// Profile layout: row c holds the stage's 16K columns as int16x2 words in
// chunks of 4 columns; chunk q of DP lane t sits at word q*64 + t*4, so the
// 8 lanes of a shared-memory phase read 8 consecutive 16-byte chunks
// whatever rows they are on (rows are multiples of 128 bytes).
template <int K>
__host__ __device__ constexpr int kp_prof_words(int A) {
  return (A + 1) * kKpG * K;
}

// Resident blocks per SM requested from ptxas: what shared memory allows for
// BLOSUM-sized alphabets (24 symbols + pad: (A+1) x 16K words of profile per
// block plus 3.7 KB of static tables and rings; 51.2 KB for K = 32, so 4
// blocks fit in the SM's 228 KB).
template <int K>
struct KPMinBlocks {
  static constexpr int value = K <= 8 ? 8 : K <= 16 ? 6 : K <= 20 ? 5 : 4;
};

template <int K>
__global__ void __launch_bounds__(32 * kKpWarps, KPMinBlocks<K>::value) kp_kernel(const __grid_constant__ KPParams p) {
  using Cell = CellS16x2;
  using T = uint32_t;
  constexpr int G = kKpG, W = G * K, kRing = 4 * G, CH = K / 4;  // CH: 4-column chunks per lane
  static_assert(K % 4 == 0, "profile rows are 16-byte chunks of 4 columns");
  extern __shared__ __align__(16) uint32_t kp_prof[];
  // sigma transposed: sigT_s[c * 32 + x] = sigma(query code x, target code c);
  // rows c >= A and columns x >= A are 0 (x = 31 is the pad column)
  __shared__ __align__(16) int8_t sigT_s[32 * 32];
  __shared__ uint8_t ring_s[kKpGroups][5 * G];  // row codes, mirrored ring
  __shared__ uint2 in_ring_s[kKpGroups][2 * G];  // left edge: the current and the next batch
  __shared__ int task_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / G, t = lane % G, grp = warp * 2 + g;
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
    const int c = i >> 5, x = i & 31;
    sigT_s[i] = (c < p.A && x < p.A) ? p.sigma[x * p.A + c] : (int8_t)0;
  }
  uint8_t *ring = ring_s[grp];
  uint2 *in_ring = in_ring_s[grp];
  int2 *bnd = p.bnd + (size_t)(blockIdx.x * kKpGroups + grp) * (size_t)p.bnd_stride;
  const int A = p.A, alpha = p.alpha, beta = p.beta;
  const T NB = Cell::splat(-beta), NAc = Cell::splat(-alpha);
  const int ngroups = (p.ntv + kKpGroups - 1) / kKpGroups;
  const int nqp = (p.nqb + 1) / 2;
  const int64_t ntasks = (int64_t)nqp * ngroups;
  int cur_qp = -1, cur_stage = -1;  // query pair and stage of the profile

  for (;;) {
    __syncthreads();  // the previous task is done everywhere (and sigT_s is filled)
    if (threadIdx.x == 0) task_s = atomicAdd(p.task_counter, 1);
    __syncthreads();
    const int task = task_s;
    if ((int64_t)task >= ntasks) break;
    const int qp = task / ngroups, tg = task % ngroups;
    int kq[2], m[2];
    int64_t qs[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int qi = 2 * qp + h;
      kq[h] = qi < p.nqb ? p.queries[qi] : -1;
      qs[h] = kq[h] >= 0 ? p.q_off[kq[h]] : 0;
      m[h] = kq[h] >= 0 ? (int)(p.q_off[kq[h] + 1] - qs[h]) : 0;
    }
    const int slot = tg * kKpGroups + grp;
    const int tid = slot < p.ntv ? p.t_sorted[slot] : -1;
    const int64_t tstart = tid >= 0 ? p.t_off[tid] : 0;
    const int len = tid >= 0 ? (int)(p.t_off[tid + 1] - tstart) : 0;
    // the target's first packed word and its position in it: row r's code is
    // residue trem + r - 1 of the words from tword on (32-bit arithmetic)
    const uint32_t *tword = p.t_packed5 + tstart / 6;
    const int trem = (int)(tstart % 6);
    const int Rw = __reduce_max_sync(0xffffffffu, (unsigned)len);  // rows of this warp
    const int nstage = (::max(m[0], m[1]) + W - 1) / W;            // the same for the whole block
    T best = Cell::splat(0);

    for (int s = 0; s < nstage; ++s) {
      // ---- the block's profile of this stage's columns ------------------
      if (qp != cur_qp || s != cur_stage) {
        __syncthreads();  // nobody reads the old profile any more
        for (int ch = threadIdx.x; ch < W / 4; ch += blockDim.x) {
          const int dt = ch / CH, q = ch - dt * CH;  // DP lane and its chunk
          const int col0 = s * W + dt * K + 4 * q;
          int x0[4], x1[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            x0[i] = col0 + i < m[0] ? (int)p.q_codes[qs[0] + col0 + i] : 31;
            x1[i] = col0 + i < m[1] ? (int)p.q_codes[qs[1] + col0 + i] : 31;
          }
          uint4 *dst = reinterpret_cast<uint4 *>(kp_prof + q * 64 + dt * 4);
          for (int c = 0; c <= A; ++c) {
            const int8_t *row = sigT_s + c * 32;
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              w[i] = (uint32_t)(uint16_t)(int16_t)row[x0[i]] | ((uint32_t)(uint16_t)(int16_t)row[x1[i]] << 16);
            dst[(size_t)c * (W / 4)] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        cur_qp = qp;
        cur_stage = s;
        __syncthreads();
      }
      if (Rw == 0) continue;  // a warp past the last target
      // ---- row codes, refilled G rows ahead -----------------------------
      auto fill_batch = [&](int b) {
        const int r = b * G + 1 + t;
        uint8_t c = (uint8_t)A;
        if (r <= len) {
          const unsigned x = (unsigned)(trem + r - 1), wq = x / 6u;
          c = (uint8_t)((__ldg(tword + wq) >> (5u * (x - 6u * wq))) & 31u);
        }
        const int sl = r & (kRing - 1);
        ring[sl] = c;
        if (sl < G) ring[sl + kRing] = c;
      };
      // left edge of the stage, batched (rows 16b+1 .. 16b+16); batch b is
      // loaded while lane 0 still reads batch b-1, and before lane 15
      // overwrites those rows with this stage's right edge (15 rows later)
      auto load_edge = [&](int b) {
        if (s > 0) {
          const int r = b * G + 1 + t;
          if (r <= Rw) {
            const int2 v = bnd[r];
            in_ring[(r - 1) & (2 * G - 1)] = make_uint2((uint32_t)v.x, (uint32_t)v.y);
          }
        }
      };
      const bool edge_out = s + 1 < nstage;
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
          const uint2 v = in_ring[(r - 1) & (2 * G - 1)];
          hl = v.x;
          fl = v.y;
        }
      };
      T Hdiag = Cell::splat(0), Hleft = Cell::splat(0), Fin = Cell::splat(CellInfo<Cell>::kNeg);
      if (t == 0) left(1, Hleft, Fin);
      const uint32_t *plane = kp_prof + t * 4;

      // One row step of this lane.  GENERAL: some lane of the group is
      // outside rows 1..Rw or lane 0's next edge row is past Rw; the other
      // batches of G steps run without those checks.
      const int nit = Rw + G - 1;
      auto step = [&](int it, uint32_t rc, auto general_tag) {
        constexpr bool GENERAL = decltype(general_tag)::value;
        const int r = it - t + 1;
        // lane 0's next left input, read before the row update
        T hl = Cell::splat(0), fl = NAc;
        if (t == 0 && (!GENERAL || it + 2 <= Rw)) left(it + 2, hl, fl);
        T Hout = H[K - 1], Fout = Cell::splat(CellInfo<Cell>::kNeg);
        if (!GENERAL || (unsigned)(r - 1) < (unsigned)Rw) {
          const uint4 *pr = reinterpret_cast<const uint4 *>(plane + (size_t)rc * W);
          uint32_t w[K];
#pragma unroll
          for (int q = 0; q < CH; ++q) {
            const uint4 a = pr[q * 16];
            w[4 * q] = a.x; w[4 * q + 1] = a.y; w[4 * q + 2] = a.z; w[4 * q + 3] = a.w;
          }
          Fout = dp_row<Cell, kModeLocal, K>(
              H, E, Hdiag, Fin, NB, best, [&](int j) -> T { return w[j]; }, [&](int) -> T { return NAc; });
          Hout = H[K - 1];
          if (t == G - 1 && edge_out) bnd[r] = make_int2((int)Hout, (int)Fout);
        }
        Hdiag = Hleft;
        Hleft = __shfl_up_sync(0xffffffffu, Hout, 1, G);
        Fin = __shfl_up_sync(0xffffffffu, Fout, 1, G);
        if (t == 0) {
          Hleft = hl;
          Fin = fl;
        }
      };
      for (int it0 = 0; it0 < nit; it0 += G) {
        __syncwarp();
        fill_batch(it0 / G + 2);
        load_edge(it0 / G + 1);
        __syncwarp();
        // this lane's ring entries of the batch are contiguous (mirrored ring)
        const uint8_t *rp = ring + ((it0 - t + 1) & (kRing - 1));
        if (it0 >= G - 1 && it0 + G + 1 <= Rw) {
#pragma unroll 2
          for (int k = 0; k < G; ++k) step(it0 + k, rp[k], std::false_type{});
        } else {
          const int nb = ::min(G, nit - it0);
          for (int k = 0; k < nb; ++k) step(it0 + k, rp[k], std::true_type{});
        }
      }
      __syncwarp();  // the edge stores are ordered before the next stage's loads
    }

    // ---- scores ----------------------------------------------------------
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = group_max<G>(cell_get<Cell>(best, h));
      if (kq[h] >= 0 && tid >= 0 && t == 0) {
        const int64_t pid = (int64_t)kq[h] * p.nt + tid;
        if (v >= 32767 - p.sigma_max_pos) {
          p.scores[pid] = kRerunMark;
          const int sl = atomicAdd(p.rerun_count, 1);
          if (sl < p.rerun_cap) p.rerun_list[sl] = (int32_t)pid;
        } else {
          p.scores[pid] = v;
        }
      }
    }
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

// Ids of up to `cap` score entries that still hold kRerunMark (pairs flagged
// for the int32 rerun after the rerun list overflowed); *count receives the
// number of marked entries found, which may exceed cap.
__global__ void kp_collect_marked_kernel(const int32_t *scores, int64_t total, int32_t *list, int32_t cap,
                                         int32_t *count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (scores[i] == kRerunMark) {
      const int sl = atomicAdd(count, 1);
      if (sl < cap) list[sl] = (int32_t)i;
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
