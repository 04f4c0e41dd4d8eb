// ga_inter.cuh -- inter-sequence DP kernel: one pair per group of G lanes,
// two pairs per lane with packed int16x2 cells.
//
// Mapping (Sec. 3.1, "Mapping Matrix Cells and Sequences to Threads"): a
// group of G lanes computes one alignment (int32) or two alignments packed
// into the low/high int16 halves of each register (int16x2, the exact
// integer counterpart of the paper's half2 packing, Sec. 3.2).  Lane t owns
// K adjacent columns of the shorter sequence; the wavefront advances one
// row (residue of the longer sequence) per iteration and lane t works on
// row it - t + 1, receiving H/F of the column left of its tile from lane
// t-1 with __shfl_up_sync.  A pair takes R + G - 1 iterations.
//
// Substitution scores (alphabets of <= 4 symbols): instead of a scoring
// profile in shared memory (Sec. 3.1) each lane keeps one byte-permute
// selector per column; the per-row "table word" holds sigma(row residue, c)
// for the four column residues c as bytes, so one prmt yields the packed,
// sign-extended sigma of both pairs.  Table words for the next rows sit in
// a per-group shared-memory ring of 4G rows refilled every G iterations
// (the counterpart of the paper's coalesced query reload every p
// iterations).
//
// Padding: columns beyond a pair's width use a selector that replicates a
// table byte's sign (sigma in {0,-1}), rows beyond its length an all-zero
// table word; pad cells never exceed the real maximum, and no real cell
// depends on a pad cell.  Results:
//   global -- H(m,n), read by the lane owning column n when it reaches row m;
//   semi   -- gaps leaving the last real column cost 0, which turns H(i,n)
//             into the running max of the last column; the score is the
//             max over row m (pad columns are <= that max) and 0;
//   local  -- running max over every cell; int16 results that reach
//             32767 - sigma_max are queued for an exact int32 rerun.
#pragma once

#include "ga_dp.cuh"

namespace ga {

struct KAParams {
  const uint32_t *packed_q;  // 2-bit codes, sequence k starts at word q_off[k]/16 + k
  const uint32_t *packed_t;
  const int64_t *q_off;
  const int64_t *t_off;
  const int4 *info;          // per pair: rows R, cols C, swap, class
  const int32_t *sorted;     // pair ids in (class, bin, R desc) order
  const int32_t *range;      // [start, end) of this bin in `sorted`
  int32_t *task_counter;     // dynamic task queue
  uint32_t tables[16];       // [0..4] table words by row code (4 = pad) for
                             // unswapped pairs, [8..12] for swapped pairs
  int32_t alpha, beta;
  int32_t sigma_max_pos;     // max(sigma_max, 0)
  int32_t *scores;
  int32_t *rerun_list;       // pair ids to recompute in int32 (local overflow)
  int32_t *rerun_count;
  int64_t nt, q0;            // cross chunk: pair p = (q0 + p/nt, p%nt); batch: nt = 0
};

template <class Cell, int MODE, int G, int K>
__device__ __forceinline__ void ka_run_task(const KAParams &p, int lane, int task,
                                            uint2 *ring /* [4G] of this group */) {
  using T = typename Cell::T;
  constexpr bool kPacked = CellInfo<Cell>::kPacked;
  constexpr int kHalves = CellInfo<Cell>::kHalves;
  constexpr int kGroups = 32 / G;
  constexpr int kPairsPerTask = kHalves * kGroups;
  constexpr int kRing = 4 * G;
  constexpr int kNeg = CellInfo<Cell>::kNeg;

  const int g = lane / G;
  const int t = lane % G;
  const int end = p.range[1];
  const int base = p.range[0] + task * kPairsPerTask;

  // ---- the pairs of this group (half 0 = low, half 1 = high) ----------
  int id[2] = {-1, -1}, R[2] = {0, 0}, C[2] = {0, 0}, sw[2] = {0, 0};
  int64_t roww[2] = {0, 0}, colw[2] = {0, 0};
#pragma unroll
  for (int h = 0; h < kHalves; ++h) {
    int s = base + g * kHalves + h;
    if (s < end) {
      int pid = p.sorted[s];
      int4 inf = p.info[pid];
      id[h] = pid; R[h] = inf.x; C[h] = inf.y; sw[h] = inf.z;
      const int64_t qi = p.nt ? p.q0 + pid / p.nt : pid, ti = p.nt ? pid % p.nt : pid;
      const int64_t qw = p.q_off[qi] / 16 + qi, tw = p.t_off[ti] / 16 + ti;
      roww[h] = sw[h] ? tw : qw;  // rows: the longer sequence
      colw[h] = sw[h] ? qw : tw;
    }
  }
  const uint32_t *rowbase[2], *colbase[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    rowbase[h] = sw[h] ? p.packed_t : p.packed_q;
    colbase[h] = sw[h] ? p.packed_q : p.packed_t;
  }
  const int Rtask = __reduce_max_sync(0xffffffffu, (unsigned)max(R[0], R[1]));

  // ---- per-column selectors, per-column gap open (semi), row 0 ---------
  const int alpha = p.alpha, beta = p.beta;
  T sel[K];
  T na[MODE == kModeSemi ? K : 1];
  T H[K], E[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int col = t * K + j;  // 0-based column index
    uint32_t s = 0;
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      const int c = (col < C[h]) ? packed_code(colbase[h], colw[h], col) : -1;
      if constexpr (kPacked) {
        const uint32_t n0 = (c >= 0) ? (uint32_t)(c + 4 * h) : (uint32_t)(8 + 4 * h);
        const uint32_t n1 = (c >= 0) ? (uint32_t)(c + 4 * h + 8) : (uint32_t)(8 + 4 * h);
        s |= (n0 | (n1 << 4)) << (8 * h);
      } else {
        const uint32_t n0 = (c >= 0) ? (uint32_t)c : 8u;
        const uint32_t n1 = (c >= 0) ? (uint32_t)(c + 8) : 8u;
        s = n0 | (n1 << 4) | (n1 << 8) | (n1 << 12);
      }
    }
    sel[j] = (T)s;
    if constexpr (MODE == kModeSemi) {
      const int a0 = (col == C[0] - 1) ? 0 : -alpha;
      const int a1 = (col == C[1] - 1) ? 0 : -alpha;
      if constexpr (kPacked) na[j] = (T)pack2(a0, a1);
      else na[j] = (T)a0;
    }
    int h0 = 0;
    if constexpr (MODE == kModeGlobal) h0 = ::max(-alpha - beta * col, kNeg);  // H(0, col+1)
    H[j] = Cell::splat(h0);
    // E holds E(i, .) of the row about to be computed: E(1, j) =
    // max(E(0, j) - beta, H(0, j) - alpha) with E(0, j) = -inf.
    E[j] = Cell::splat(::max(h0 - alpha, kNeg));
  }
  // Lane 0 starts row 1 at iteration 0 with H(1,0) on its left and H(0,0)=0
  // on its diagonal.  Lane t > 0 starts row 1 at iteration t; its diagonal
  // is the left tile's row-0 value H(0, t*K), which Hleft carries until the
  // first shuffle replaces it.
  int hd0 = 0;
  if constexpr (MODE == kModeGlobal) hd0 = (t == 0) ? 0 : ::max(-alpha - beta * (t * K - 1), kNeg);
  const int hb0 = (MODE == kModeGlobal) ? -alpha : 0;  // H(1,0)
  T Hdiag = Cell::splat(hd0);
  T Hleft = Cell::splat(t == 0 ? hb0 : hd0);
  // Lane 0's F(r, 1) = max(F(r, 0) - beta, H(r, 0) - alpha), F(r, 0) = -inf.
  T Fin = Cell::splat(t == 0 ? hb0 - alpha : kNeg);
  T hb = Cell::splat(hb0);  // lane 0: H(r,0) of its current row
  const T nbeta_b = Cell::splat((MODE == kModeGlobal) ? -beta : 0);
  const T NAc = Cell::splat(-alpha);
  const T NB = Cell::splat(-beta);
  const T NEGV = Cell::splat(kNeg);
  T best = Cell::splat(0);
  int res[2] = {0, 0};
  bool got[2] = {false, false};

  // ---- row table words: ring of 4G rows, refilled a batch of G ahead --
  auto table_word = [&](int h, int r) -> uint32_t {
    if (r > R[h] || r < 1) return 0u;
    const int code = packed_code(rowbase[h], roww[h], r - 1);
    return p.tables[(sw[h] ? 8 : 0) + code];
  };
  auto fill_batch = [&](int b) {
    const int r = b * G + 1 + t;
    uint2 v;
    v.x = table_word(0, r);
    v.y = kPacked ? table_word(1, r) : 0u;
    ring[r & (kRing - 1)] = v;
  };
  fill_batch(0);
  fill_batch(1);
  __syncwarp();

  const int nit = Rtask + G - 1;
  for (int it = 0; it < nit; ++it) {
    if ((it % G) == 0) {
      fill_batch(it / G + 2);  // rows needed from iteration it + 2G on
      __syncwarp();
    }
    const int r = it - t + 1;
    T Hout, Fout;
    if ((unsigned)(r - 1) < (unsigned)Rtask) {
      const uint2 tw = ring[r & (kRing - 1)];
      Fout = dp_row<Cell, MODE, K>(
          H, E, Hdiag, Fin, NB, best,
          [&](int j) -> T { return (T)prmt(tw.x, tw.y, (uint32_t)sel[j]); },
          [&](int j) -> T {
            if constexpr (MODE == kModeSemi) return na[j];
            else return NAc;
          });
      Hout = H[K - 1];
      if constexpr (MODE != kModeLocal) {
        if (r == R[0] || r == R[1]) {
#pragma unroll
          for (int h = 0; h < kHalves; ++h) {
            if (r != R[h]) continue;
            if constexpr (MODE == kModeGlobal) {
              const int o = C[h] - 1 - t * K;  // column n in this tile?
              if (o >= 0 && o < K) {
                T v = H[0];
#pragma unroll
                for (int j = 1; j < K; ++j)
                  if (j == o) v = H[j];
                res[h] = cell_get<Cell>(v, h);
                got[h] = true;
              }
            } else {
              int mx = 0;
#pragma unroll
              for (int j = 0; j < K; ++j) mx = ::max(mx, cell_get<Cell>(H[j], h));
              res[h] = mx;
            }
          }
        }
      }
    } else {
      Hout = H[K - 1];
      Fout = NEGV;
    }
    Hdiag = Hleft;
    Hleft = __shfl_up_sync(0xffffffffu, Hout, 1, G);
    Fin = __shfl_up_sync(0xffffffffu, Fout, 1, G);
    hb = Cell::add(hb, nbeta_b);
    if (t == 0) {
      Hleft = hb;
      Fin = Cell::add(hb, NAc);
    }
  }

  // ---- results ----------------------------------------------------------
#pragma unroll
  for (int h = 0; h < kHalves; ++h) {
    int v = 0;
    if constexpr (MODE == kModeLocal) v = group_max<G>(cell_get<Cell>(best, h));
    else if constexpr (MODE == kModeSemi) v = group_max<G>(res[h]);
    else v = res[h];
    if (id[h] < 0) continue;
    if constexpr (MODE == kModeGlobal) {
      if (got[h]) p.scores[id[h]] = v;
    } else if (t == 0) {
      if (kPacked && MODE == kModeLocal && v >= 32767 - p.sigma_max_pos) {
        const int slot = atomicAdd(p.rerun_count, 1);
        p.rerun_list[slot] = id[h];
      } else {
        p.scores[id[h]] = v;
      }
    }
  }
}

template <class Cell, int MODE, int G, int K>
__global__ void __launch_bounds__(128) ka_kernel(const __grid_constant__ KAParams p) {
  constexpr int kWarps = 4;
  constexpr int kGroups = 32 / G;
  __shared__ uint2 ring_s[kWarps][kGroups][4 * G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npairs = p.range[1] - p.range[0];
  constexpr int kPairsPerTask = CellInfo<Cell>::kHalves * kGroups;
  const int ntasks = (npairs + kPairsPerTask - 1) / kPairsPerTask;
  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= ntasks) break;
    ka_run_task<Cell, MODE, G, K>(p, lane, task, ring_s[warp][lane / G]);
  }
}

}  // namespace ga
