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
  const uint32_t *packed_q;  // flat 2-bit codes: residue x in word x/16
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

// Per-group state that the hot loop needs only every G iterations (ring
// refill) or once (results) lives in shared memory, not in registers.
struct KAGroupDesc {
  const uint32_t *rowbase[2];  // packed stream holding each half's row sequence
  int64_t rowpos[2];           // position of its first residue in that stream
  int R[2];                    // rows of each half (0: no pair)
  int tab[2];                  // table word offset: 0 (rows = query) or 8
};

// Column tiles of the inter-sequence kernel: 16 lanes x K columns per pair
// (widths 96 .. 320 in steps of 16, then 384 and 512), so a pair's padding
// to its tile is at most 15 columns up to 320 columns.
constexpr int kKaNumBins = 17;
constexpr int kKaK[kKaNumBins] = {6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 24, 32};

__host__ __device__ constexpr int ka_tile_index(int K) {
  int i = 0;
  while (i < kKaNumBins - 1 && kKaK[i] < K) ++i;
  return i;
}

// Minimum resident blocks per SM requested from ptxas (__launch_bounds__):
// the highest occupancy at which each (cell type, mode, K) instantiation
// compiles on sm_103a without register spills (local mode and the int32
// cells) or with at most 16 bytes of spill stores (packed global and
// semi-global: the extra resident block measured faster on GB300, local
// measured slower).  The values come from compiling every instantiation at
// each candidate block count and reading ptxas's spill report; they must be
// re-derived the same way after a change to the kernel.
template <class Cell, int MODE, int K>
struct KAMinBlocks {
  // columns per lane:    6  7  8  9 10 11 12 13 14 15 16 17 18 19 20 24 32
  static constexpr int kPacked[3][kKaNumBins] = {
      {8, 8, 8, 6, 6, 6, 6, 6, 8, 6, 6, 5, 6, 5, 5, 4, 3},   // local (no spills)
      {8, 8, 8, 8, 8, 6, 6, 5, 5, 5, 5, 6, 5, 4, 4, 3, 1},   // global (<= 16 bytes)
      {8, 8, 8, 6, 8, 6, 6, 5, 6, 5, 5, 4, 4, 4, 4, 3, 3}};  // semi-global (<= 16 bytes)
  static constexpr int kScalar[3][kKaNumBins] = {
      {8, 8, 8, 8, 8, 6, 8, 8, 8, 6, 6, 6, 6, 6, 5, 4, 3},
      {8, 8, 8, 6, 6, 8, 6, 8, 6, 5, 6, 5, 5, 5, 5, 1, 1},
      {8, 8, 8, 8, 8, 6, 6, 6, 5, 6, 5, 4, 4, 4, 3, 3, 1}};
  static constexpr int kIdx = ka_tile_index(K);
  static constexpr int value = CellInfo<Cell>::kPacked ? kPacked[MODE][kIdx] : kScalar[MODE][kIdx];
};

template <class Cell, int MODE, int G, int K>
__device__ __forceinline__ void ka_run_task(const KAParams &p, int lane, int task,
                                            uint2 *ring /* [5G]: 4G-row ring + mirror of its first G rows */,
                                            KAGroupDesc *desc, uint32_t *evbuf /* [2][K] */) {
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
  int id[2] = {-1, -1}, R[2] = {0, 0}, C[2] = {0, 0};
  const uint32_t *colbase[2] = {p.packed_t, p.packed_t};
  int64_t colpos[2] = {0, 0};
#pragma unroll
  for (int h = 0; h < kHalves; ++h) {
    const int s = base + g * kHalves + h;
    const uint32_t *rowbase = p.packed_q;
    int64_t rowpos = 0;
    int sw = 0;
    if (s < end) {
      const int pid = p.sorted[s];
      const int4 inf = p.info[pid];
      id[h] = pid; R[h] = inf.x; C[h] = inf.y; sw = inf.z;
      const int64_t qi = p.nt ? p.q0 + pid / p.nt : pid, ti = p.nt ? pid % p.nt : pid;
      const int64_t qs = p.q_off[qi], ts = p.t_off[ti];
      rowbase = sw ? p.packed_t : p.packed_q;  // rows: the longer sequence
      rowpos = sw ? ts : qs;
      colbase[h] = sw ? p.packed_q : p.packed_t;
      colpos[h] = sw ? qs : ts;
    }
    if (t == 0) {
      desc->rowbase[h] = rowbase;
      desc->rowpos[h] = rowpos;
      desc->R[h] = R[h];
      desc->tab[h] = sw ? 8 : 0;
    }
  }
  if (kHalves == 1 && t == 0) {
    desc->rowbase[1] = p.packed_q;
    desc->rowpos[1] = 0;
    desc->R[1] = 0;
    desc->tab[1] = 0;
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
      const int c = (col < C[h]) ? packed_code(colbase[h], colpos[h] + col) : -1;
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
  // Which half ends on which row, and (global) which lane owns column n.
  const int own0 = (C[0] - 1) / K, own1 = (C[1] - 1) / K;
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
  T rmax = Cell::splat(0);  // semi: packed max over the row m of each half

  // ---- row table words: ring of 4G rows, refilled a batch of G ahead --
  // The descriptor is re-read (volatile) at every refill so that the
  // compiler cannot keep it in registers across the hot loop.
  const volatile KAGroupDesc *vdesc = desc;
  auto fill_batch = [&](int b) {
    const int r = b * G + 1 + t;
    uint2 v = make_uint2(0u, 0u);
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      if (r <= vdesc->R[h]) {
        const uint32_t tw = p.tables[vdesc->tab[h] + packed_code((const uint32_t *)vdesc->rowbase[h],
                                                                 vdesc->rowpos[h] + (r - 1))];
        if (h == 0) v.x = tw; else v.y = tw;
      }
    }
    const int slot = r & (kRing - 1);
    ring[slot] = v;
    if (slot < G) ring[slot + kRing] = v;  // mirror: any G consecutive rows are contiguous
  };
  __syncwarp();
  fill_batch(0);
  fill_batch(1);
  __syncwarp();

  // Event window: iterations in which some lane of the warp reaches the
  // last row of one of its pairs (global: read H(m,n); semi: row-m max).
  int rlo = 1 << 30, rhi = 0;
#pragma unroll
  for (int h = 0; h < kHalves; ++h)
    if (R[h] > 0) {
      rlo = ::min(rlo, R[h]);
      rhi = ::max(rhi, R[h]);
    }
  const int ev_lo = (int)__reduce_min_sync(0xffffffffu, (unsigned)rlo) - 1;
  const int ev_hi = (int)__reduce_max_sync(0xffffffffu, (unsigned)rhi) + G - 2;

  // One wavefront step.  GENERAL: lanes may be outside [1, Rtask] (the
  // first G-1 iterations) or at the last row of a pair (event window).
  // Outside those the step runs without checks: rows beyond a pair's end
  // use the all-zero table word, so the lanes that run past Rtask during
  // the drain compute pad rows that no real cell reads and that can never
  // raise a running max.
  auto step = [&](int it, const uint2 *rp, auto general_tag) {
    constexpr bool GENERAL = decltype(general_tag)::value;
    const int r = it - t + 1;
    T Hout, Fout;
    if (!GENERAL || (unsigned)(r - 1) < (unsigned)Rtask) {
      const uint2 tw = *rp;
      Fout = dp_row<Cell, MODE, K>(
          H, E, Hdiag, Fin, NB, best,
          [&](int j) -> T { return (T)prmt(tw.x, tw.y, (uint32_t)sel[j]); },
          [&](int j) -> T {
            if constexpr (MODE == kModeSemi) return na[j];
            else return NAc;
          });
      Hout = H[K - 1];
      if constexpr (GENERAL && MODE != kModeLocal) {
        if (r == R[0] || r == R[1]) {
          if constexpr (MODE == kModeGlobal) {
            // the lane owning column n parks its row in shared memory
#pragma unroll
            for (int h = 0; h < kHalves; ++h)
              if (r == R[h] && t == (h ? own1 : own0)) {
#pragma unroll
                for (int j = 0; j < K; ++j) evbuf[h * K + j] = (uint32_t)H[j];
              }
          } else {
            T m = H[0];
#pragma unroll
            for (int j = 1; j + 1 < K; j += 2) m = Cell::max3(m, H[j], H[j + 1]);
            if ((K & 1) == 0) m = Cell::max(m, H[K - 1]);
            if constexpr (kPacked) {
              const uint32_t keep = (r == R[0] ? 0x0000ffffu : 0u) | (r == R[1] ? 0xffff0000u : 0u);
              rmax = (T)(((uint32_t)Cell::max(rmax, m) & keep) | ((uint32_t)rmax & ~keep));
            } else {
              rmax = Cell::max(rmax, m);
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
    if constexpr (MODE == kModeGlobal) {
      hb = Cell::add(hb, nbeta_b);
      if (t == 0) {
        Hleft = hb;
        Fin = Cell::add(hb, NAc);
      }
    } else if (t == 0) {  // local / semi-global: H(r,0) = 0, F(r,1) = -alpha
      Hleft = Cell::splat(0);
      Fin = NAc;
    }
  };

  // Segments of warp-uniform kind between refills (every G iterations).
  const int nit = Rtask + G - 1;
  int it = 0;
  while (it < nit) {
    if ((it % G) == 0) {
      fill_batch(it / G + 2);  // rows needed from iteration it + 2G on
      __syncwarp();
    }
    int stop = ::min(nit, (it / G + 1) * G);
    bool general;
    if (it < G - 1) {
      stop = ::min(stop, G - 1);
      general = true;
    } else if (MODE != kModeLocal && it < ev_lo) {
      stop = ::min(stop, ev_lo);
      general = false;
    } else if (MODE != kModeLocal && it <= ev_hi) {
      stop = ::min(stop, ev_hi + 1);
      general = true;
    } else {
      general = false;
    }
    // this lane's ring entries of the segment are contiguous (mirrored ring)
    const uint2 *rp = ring + ((it - t + 1) & (kRing - 1));
    if (general) {
      for (; it < stop; ++it, ++rp) step(it, rp, std::true_type{});
    } else {
#pragma unroll 2
      for (; it < stop; ++it, ++rp) step(it, rp, std::false_type{});
    }
  }
  __syncwarp();

  // ---- results ----------------------------------------------------------
#pragma unroll
  for (int h = 0; h < kHalves; ++h) {
    int v = 0;
    if constexpr (MODE == kModeLocal) v = group_max<G>(cell_get<Cell>(best, h));
    else if constexpr (MODE == kModeSemi) v = group_max<G>(cell_get<Cell>(rmax, h));
    if (id[h] < 0) continue;
    if constexpr (MODE == kModeGlobal) {
      if (t == 0) {
        const uint32_t w = evbuf[h * K + (C[h] - 1) % K];
        p.scores[id[h]] = cell_get<Cell>((T)w, h);
      }
    } else if (t == 0) {
      if (kPacked && MODE == kModeLocal && v >= 32767 - p.sigma_max_pos) {
        const int slot = atomicAdd(p.rerun_count, 1);
        p.rerun_list[slot] = id[h];
      } else {
        p.scores[id[h]] = v;
      }
    }
  }
  __syncwarp();
}

template <class Cell, int MODE, int G, int K>
__global__ void __launch_bounds__(128, KAMinBlocks<Cell, MODE, K>::value) ka_kernel(const __grid_constant__ KAParams p) {
  constexpr int kWarps = 4;
  constexpr int kGroups = 32 / G;
  __shared__ uint2 ring_s[kWarps][kGroups][5 * G];
  __shared__ KAGroupDesc desc_s[kWarps][kGroups];
  __shared__ uint32_t evbuf_s[kWarps][kGroups][MODE == kModeGlobal ? 2 * K : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npairs = p.range[1] - p.range[0];
  constexpr int kPairsPerTask = CellInfo<Cell>::kHalves * kGroups;
  const int ntasks = (npairs + kPairsPerTask - 1) / kPairsPerTask;
  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= ntasks) break;
    ka_run_task<Cell, MODE, G, K>(p, lane, task, ring_s[warp][lane / G], &desc_s[warp][lane / G],
                                  evbuf_s[warp][lane / G]);
  }
}

}  // namespace ga
