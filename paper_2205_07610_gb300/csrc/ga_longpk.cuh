// ga_longpk.cuh -- packed int16x2 kernel for long pairs over alphabets of
// <= 4 symbols: one warp per pair, two column halves of the pair in the two
// int16 halves of every register, every cell exact at any sequence length.
//
// Mapping.  The columns (shorter sequence) are cut into super-stages of
// 2 x 32 x K columns computed left to right (the multi-stage partitioning of
// Sec. 3.1).  Within a super-stage lane t owns K columns of the left half
// (low int16 halves) and the K columns 32K further right (high halves).  The
// low half of lane t works on row it - t + 1 as in the other wavefront
// kernels; the high half runs 32 rows behind, so that lane 0's high half
// receives, one iteration after lane 31's low half produced it, the H / F of
// the column left of the right half.  A single rotating __shfl_sync carries
// both halves between neighbours: lane 0 puts the left edge of the
// super-stage (the previous super-stage's right edge, from a per-warp global
// buffer batched through shared memory, or column 0) into its low half and
// lane 31's low half into its high half.  Lane 31's high half produces the
// right edge.  Substitution scores come from one prmt per packed column as
// in the inter-sequence kernel: per-column selectors and one table word per
// row for each half.
//
// Exact int16 at any length (relative values).  Each lane keeps, per half,
// an int32 base b and stores every H, E, F as the int16 difference to b.
// Adjacent cells differ by at most sigma_max + alpha (a cell is at least its
// left or upper neighbour minus alpha through a gap, and at most its
// diagonal neighbour plus sigma_max, which is itself at most alpha below the
// neighbour), so within a lane's K columns, within the rows run since its
// base was set and across one lane boundary the differences stay inside
// int16 with room for -inf (-32000) when (sigma_max + alpha) * (kKwRenorm +
// 2K + 8) < 32000 - 256 (drift over the rows since the last renormalisation,
// spread over the K columns, base difference to the neighbour, E and F below
// H).  Every
// kKwRenorm iterations each lane moves its base to its current H of its first
// column (all lanes at the same iteration) and the lanes exchange their
// bases; a value received from the left neighbour is converted with one
// packed add of the base difference D.  Absolute int32 values appear only at
// the super-stage edges and in the results.
//
// Local mode: the zero of Eq. H becomes Z = -b per half (saturated at -inf
// once b is large, where it can no longer bind), folded into E:
// E'(i,j) = max(E(i,j), Z) satisfies E'(i+1,j) = max(E'(i,j) - beta,
// H(i,j) - alpha, Z) because beta > 0, so H = max(H_diag + sigma, E', F) is
// Eq. H with nu = 0.  The running maximum is kept relative and folded into
// an int32 maximum at every renormalisation.
//
// Rows outside a half's range: before its first row the high half sees a
// "virtual" row whose table word leaves the row-0 state unchanged (sigma = 0
// for local / semi-global; -beta for global, where H(0, j) = H(0, j-1) -
// beta for the high half's columns j >= 2); after its last row a half runs
// pad rows (sigma = 0) that no real cell depends on and that never exceed
// the largest real cell; lane 0's low half then receives -inf.
#pragma once

#include "ga_dp.cuh"
#include "ga_long.cuh"

namespace ga {

constexpr int kKwRenorm = 128;  // iterations between base renormalisations
// Largest sigma_max + alpha of the packed long kernel: 128 * (128 + 2K + 8)
// = 23552 for K <= 24 keeps every relative value inside int16 with room for
// -inf.
constexpr int kKwMaxStep = 128;

__device__ __forceinline__ uint32_t pk16(int lo, int hi) {
  return (uint32_t)(lo & 0xffff) | ((uint32_t)hi << 16);
}

// Row update on relative packed cells.  As dp_row, except that local mode
// takes the zero of Eq. H from E' (see above) instead of a ReLU at 0.
template <int MODE, int K, class SigFn, class NaFn>
__device__ __forceinline__ uint32_t pk_row(uint32_t (&H)[K], uint32_t (&E)[K], uint32_t Hdiag, uint32_t Fin,
                                           uint32_t NB, uint32_t Z, uint32_t &best, SigFn SIG, NaFn NA) {
#pragma unroll
  for (int j = K - 1; j >= 1; --j) H[j] = __vadd2(H[j - 1], SIG(j));
  H[0] = __vadd2(Hdiag, SIG(0));
  uint32_t F = Fin;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    H[j] = __vimax3_s16x2(H[j], E[j], F);
    const uint32_t A = __vadd2(H[j], NA(j));
    if constexpr (MODE == kModeLocal) E[j] = __vimax3_s16x2(__vadd2(E[j], NB), A, Z);
    else E[j] = __viaddmax_s16x2(E[j], NB, A);
    F = __viaddmax_s16x2(F, NB, A);
    if constexpr (MODE == kModeLocal) {
      if ((j & 1) == 1) best = __vimax3_s16x2(best, H[j - 1], H[j]);
      else if (j == K - 1) best = __vmaxs2(best, H[j]);
    }
  }
  return F;
}

// The same row update with a one-op chain across the columns (local and
// global mode, where every column's gap open alpha >= beta).  With X(j) =
// max(Hdiag + sigma, E') the H of a column is max(X(j), F(j)), and since
// F(j) - alpha <= F(j) - beta the gap entering the next column is
// F(j+1) = max(F(j) - beta, X(j) - alpha): it no longer waits for H(j).
// One more ALU and one more FMA op per packed column than pk_row, for a
// dependency chain of one op per column instead of three: faster where a
// warp's row step is set by its latency (a scheduler with one warp), slower
// where the issue slots are shared.
template <int MODE, int K, class SigFn>
__device__ __forceinline__ uint32_t pk_row_fc(uint32_t (&H)[K], uint32_t (&E)[K], uint32_t Hdiag, uint32_t Fin,
                                              uint32_t NB, uint32_t NAc, uint32_t Z, uint32_t &best,
                                              SigFn SIG) {
  static_assert(MODE != kModeSemi, "semi-global frees the last column's gap open");
#pragma unroll
  for (int j = K - 1; j >= 1; --j) H[j] = __vadd2(H[j - 1], SIG(j));
  H[0] = __vadd2(Hdiag, SIG(0));
  uint32_t F = Fin;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const uint32_t X = __vmaxs2(H[j], E[j]);
    const uint32_t Fj = F;
    F = __viaddmax_s16x2(F, NB, __vadd2(X, NAc));
    H[j] = __vmaxs2(X, Fj);
    const uint32_t A = __vadd2(H[j], NAc);
    if constexpr (MODE == kModeLocal) E[j] = __vimax3_s16x2(__vadd2(E[j], NB), A, Z);
    else E[j] = __viaddmax_s16x2(E[j], NB, A);
    if constexpr (MODE == kModeLocal) {
      if ((j & 1) == 1) best = __vimax3_s16x2(best, H[j - 1], H[j]);
      else if (j == K - 1) best = __vmaxs2(best, H[j]);
    }
  }
  return F;
}

template <int MODE, int K>
__global__ void __launch_bounds__(128) kw_kernel(const __grid_constant__ KBParams p) {
  static_assert(kKwMaxStep * (kKwRenorm + 2 * K + 8) < 32000 - 256, "relative int16 cells of this tile width");
  constexpr int kWarps = 4;
  constexpr int WH = 32 * K;  // columns per half
  constexpr int W2 = 2 * WH;  // columns per super-stage
  constexpr int kRing = 256;  // row table words, rows r & 255 (+ a mirror of the first 32 entries)

  __shared__ int2 in_ring_s[kWarps][64];
  __shared__ int2 out_ring_s[kWarps][32];
  __shared__ uint32_t row_ring_s[kWarps][kRing + 32];

  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  int2 *in_ring = in_ring_s[warp];
  int2 *out_ring = out_ring_s[warp];
  uint32_t *row_ring = row_ring_s[warp];
  int2 *bnd = p.bnd + (size_t)(blockIdx.x * kWarps + warp) * (size_t)p.bnd_stride;

  const int npairs = p.range[1] - p.range[0];
  const int alpha = p.alpha, beta = p.beta;
  const uint32_t NB = pk16(-beta, -beta);
  const uint32_t NAc = pk16(-alpha, -alpha);
  const uint32_t NEGV = pk16(kNeg16, kNeg16);
  // table word of the virtual rows before a half's first row
  const uint32_t virt_w = (MODE == kModeGlobal) ? 0x01010101u * (uint32_t)(uint8_t)(-beta) : 0u;
  // row-0 value H(0, c) of 1-based column c (c = 0: the corner)
  auto h0 = [&](int c) -> int { return (MODE == kModeGlobal && c > 0) ? -alpha - beta * (c - 1) : 0; };

  for (;;) {
    int task = 0;
    if (t == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= npairs) break;

    const int pid = p.sorted[p.range[0] + task];
    const int4 inf = p.info[pid];
    const int R = inf.x, C = inf.y, sw = inf.z;
    const int64_t qi = p.nt ? p.q0 + pid / p.nt : pid, ti = p.nt ? pid % p.nt : pid;
    const int64_t qs = p.q_off[qi], ts = p.t_off[ti];
    const int64_t rowpos = sw ? ts : qs;
    const int64_t colpos = sw ? qs : ts;
    const uint32_t *rowbase = sw ? p.packed_t : p.packed_q;
    const uint32_t *colbase = sw ? p.packed_q : p.packed_t;
    const uint32_t *tab = p.tables + (sw ? 8 : 0);

    const int nst = (C + W2 - 1) / W2;
    int best_abs = 0;            // local: max over both halves and all stages
    int rowmax = 0;              // semi: max over row R (and column C through the free gaps)
    int gscore = 0;
    bool got = false;

    for (int s = 0; s < nst; ++s) {
      const int col0 = s * W2;
      // ---- columns, bases and row 0 of both halves ----------------------
      int b[2];                          // int32 base per half
      b[0] = h0(col0 + t * K + 1);
      b[1] = h0(col0 + WH + t * K + 1);
      uint32_t sel[K];
      uint32_t na[MODE == kModeSemi ? K : 1];
      uint32_t H[K], E[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        uint32_t sv = 0;
        int nav[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = col0 + h * WH + t * K + j;  // 0-based
          const int c = (col < C) ? packed_code(colbase, colpos + col) : -1;
          const uint32_t n0 = (c >= 0) ? (uint32_t)(c + 4 * h) : (uint32_t)(8 + 4 * h);
          const uint32_t n1 = (c >= 0) ? (uint32_t)(c + 4 * h + 8) : (uint32_t)(8 + 4 * h);
          sv |= (n0 | (n1 << 4)) << (8 * h);
          nav[h] = (col == C - 1) ? 0 : -alpha;
        }
        sel[j] = sv;
        if constexpr (MODE == kModeSemi) na[j] = pk16(nav[0], nav[1]);
        const int hv = (MODE == kModeGlobal) ? -beta * j : 0;  // H(0, first + j) - b
        H[j] = pk16(hv, hv);
        const int ev = (MODE == kModeLocal) ? 0 : hv - alpha;   // local: E' = max(E, 0) = 0
        E[j] = pk16(ev, ev);
      }
      uint32_t Z = 0;  // local: the zero of Eq. H relative to the bases (both 0 here)
      // base difference to the left neighbour (lane 0: low half unused,
      // high half against lane 31's low half)
      uint32_t D = pk16(t == 0 ? 0 : h0(col0 + t * K + 1 - K) - b[0], h0(col0 + WH + t * K + 1 - K) - b[1]);
      const int ocol = C - 1 - col0;                  // 0-based column C in this super-stage
      const int ohalf = ocol >= WH ? 1 : 0;
      const int olane = (ocol - ohalf * WH) / K, oj = (ocol - ohalf * WH) % K;
      const bool owner = (s == nst - 1) && t == olane;
      uint32_t best = 0;

      auto left_row = [&](int r) -> int2 {  // (H(r, col0), F(r, col0 + 1)), absolute
        int2 v;
        if (s == 0) {
          v.x = (MODE == kModeGlobal) ? ((r == 0) ? 0 : -alpha - beta * (r - 1)) : 0;
          v.y = v.x - alpha;
        } else {
          v = in_ring[(r - 1) & 63];
        }
        return v;
      };
      auto load_batch = [&](int bb) {  // left edge rows 32bb+1 .. 32bb+32
        if (s > 0) {
          const int r = 32 * bb + 1 + t;
          in_ring[(r - 1) & 63] = bnd[r];
        }
      };
      // table words of rows 32bb+1 .. 32bb+32 (0 for the pad rows past R):
      // read_rows loads the packed word a batch before put_rows stores the
      // table word, so the load's latency overlaps a batch of rows; the
      // ring's first 32 entries are mirrored after the last, so that the 32
      // rows a lane reads in a batch are contiguous
      auto read_rows = [&](int bb) -> uint32_t {
        const int r = 32 * bb + 1 + t;
        return (r <= R) ? __ldg(rowbase + ((rowpos + r - 1) >> 4)) : 0u;
      };
      auto put_rows = [&](int bb, uint32_t w) {
        const int r = 32 * bb + 1 + t;
        const uint32_t v = (r <= R) ? tab[(w >> (2 * (int)((rowpos + r - 1) & 15))) & 3u] : 0u;
        const int x = r & (kRing - 1);
        row_ring[x] = v;
        if (x < 32) row_ring[x + kRing] = v;
      };
      row_ring[(-t) & (kRing - 1)] = virt_w;  // rows 0 .. -31
      if (t == 0) row_ring[kRing] = virt_w;
      load_batch(0);
      put_rows(0, read_rows(0));
      put_rows(1, read_rows(1));
      uint32_t next_rows = read_rows(2);  // stored at iteration 0
      __syncwarp();

      // inputs of each half's first row: diagonal H(0, first - 1); left the
      // same (carried until the first shuffle replaces it), except lane 0's
      // low half, whose left input is the super-stage's edge at row 1
      const int hd0 = h0(col0 + t * K) - b[0], hd1 = h0(col0 + WH + t * K) - b[1];
      uint32_t Hdiag = pk16(hd0, hd1);
      uint32_t Hleft = Hdiag;
      uint32_t Fin = NEGV;
      if (t == 0) {
        const int2 l1 = left_row(1);
        Hleft = pk16(l1.x - b[0], hd1);
        Fin = pk16(l1.y - b[0], kNeg16);
      }

      // Lane 31's high-half output rows are kept as raw packed words and
      // turned into absolute edge values when they are flushed, with lane
      // 31's high-half base: every batch flushes all rows stored before it,
      // ahead of any renormalisation.
      auto flush_rows = [&](int first, int last_row) {  // at most 32 rows, lane t: row first + t
        const int b31 = __shfl_sync(0xffffffffu, b[1], 31);
        const int r = first + t;
        if (r <= last_row) {
          const int2 o = out_ring[(r - 1) & 31];
          bnd[r] = make_int2(hi16((uint32_t)o.x) + b31, hi16((uint32_t)o.y) + b31);
        }
      };

      // One row step of this lane.  GENERAL: some lane of the warp is before
      // row 1, past row R or at row R, lane 31's output row or lane 0's next
      // edge row is outside 1..R; the other batches of 32 steps run without
      // checks.
      auto step = [&](int it, uint32_t twl, uint32_t twh, auto general_tag) {
        constexpr bool GENERAL = decltype(general_tag)::value;
        // lane 0's next left input (the edge at row it + 2), read before the
        // row update so that it is ready when the shuffles are
        int lx = kNeg16, ly = kNeg16;
        if (t == 0 && (!GENERAL || it + 2 <= R)) {
          const int2 lv = left_row(it + 2);
          lx = lv.x - b[0];
          ly = lv.y - b[0];
        }
        const int rlo = it - t + 1, rhi = rlo - 32;
        uint32_t Hout, Fout;
        if (!GENERAL || rlo >= 1) {
          Fout = pk_row<MODE, K>(
              H, E, Hdiag, Fin, NB, Z, best, [&](int j) -> uint32_t { return prmt(twl, twh, sel[j]); },
              [&](int j) -> uint32_t {
                if constexpr (MODE == kModeSemi) return na[j];
                else return NAc;
              });
          Hout = H[K - 1];
          if constexpr (GENERAL && MODE != kModeLocal) {
            if (rlo == R || rhi == R) {
              const int h = (rhi == R) ? 1 : 0;
              if constexpr (MODE == kModeGlobal) {
                if (owner && h == ohalf) {
                  uint32_t v = H[0];
#pragma unroll
                  for (int j = 1; j < K; ++j)
                    if (j == oj) v = H[j];
                  gscore = h ? hi16(v) + b[1] : lo16(v) + b[0];
                  got = true;
                }
              } else {
                uint32_t m = H[0];
#pragma unroll
                for (int j = 1; j < K; ++j) m = __vmaxs2(m, H[j]);
                rowmax = ::max(rowmax, h ? hi16(m) + b[1] : lo16(m) + b[0]);
              }
            }
          }
        } else {
          Hout = H[K - 1];
          Fout = NEGV;
        }
        if (t == 31 && (!GENERAL || (rhi >= 1 && rhi <= R)))
          out_ring[(rhi - 1) & 31] = make_int2((int)Hout, (int)Fout);
        Hdiag = Hleft;
        uint32_t hs = __shfl_sync(0xffffffffu, Hout, (t + 31) & 31);
        uint32_t fs = __shfl_sync(0xffffffffu, Fout, (t + 31) & 31);
        if (t == 0) {  // low half: the edge's next row; high half: lane 31's low half
          hs = prmt((uint32_t)lx, hs, 0x5410u);
          fs = prmt((uint32_t)ly, fs, 0x5410u);
        }
        Hleft = __vadd2(hs, D);
        Fin = __vadd2(fs, D);
      };

      const int nit = R + 63;
      int flushed = 0;  // edge rows 1..flushed are in bnd
      for (int it0 = 0; it0 < nit; it0 += 32) {
        __syncwarp();
        load_batch(it0 / 32 + 1);
        put_rows(it0 / 32 + 2, next_rows);
        next_rows = read_rows(it0 / 32 + 3);
        if (it0 >= 64) {  // lane 31's high-half rows stored since the last flush: .. it0-63
          flush_rows(flushed + 1, it0 - 63);
          flushed = it0 - 63;
        }
        if ((it0 & (kKwRenorm - 1)) == 0 && it0 > 0) {
          // move each half's base to its current H of the first column
          const int d0 = lo16(H[0]), d1 = hi16(H[0]);
          if constexpr (MODE == kModeLocal) {
            best_abs = ::max(best_abs, ::max(lo16(best) + b[0], hi16(best) + b[1]));
            best = NEGV;
          }
          b[0] += d0;
          b[1] += d1;
          const uint32_t dl = pk16(-d0, -d1);
#pragma unroll
          for (int j = 0; j < K; ++j) {
            H[j] = __vadd2(H[j], dl);
            E[j] = __vadd2(E[j], dl);
          }
          Hdiag = __vadd2(Hdiag, dl);
          Hleft = __vadd2(Hleft, dl);
          Fin = __vadd2(Fin, dl);
          if constexpr (MODE == kModeLocal) {  // the zero of Eq. H under the new bases
            Z = pk16(::max(-b[0], kNeg16), ::max(-b[1], kNeg16));
#pragma unroll
            for (int j = 0; j < K; ++j) E[j] = __vmaxs2(E[j], Z);
          }
          const int nb0 = __shfl_sync(0xffffffffu, b[0], (t + 31) & 31);
          const int nb1 = __shfl_sync(0xffffffffu, b[1], (t + 31) & 31);
          D = (t == 0) ? pk16(0, nb0 - b[1]) : pk16(nb0 - b[0], nb1 - b[1]);
        }
        __syncwarp();
        // this lane's ring entries of the batch are contiguous (mirrored ring)
        const uint32_t *rl = row_ring + ((it0 - t + 1) & (kRing - 1));
        const uint32_t *rh = row_ring + ((it0 - t - 31) & (kRing - 1));
        if (it0 >= 64 && it0 + 33 <= R) {
#pragma unroll 2
          for (int k = 0; k < 32; ++k) step(it0 + k, rl[k], rh[k], std::false_type{});
        } else {
          const int n = ::min(32, nit - it0);
          for (int k = 0; k < n; ++k) step(it0 + k, rl[k], rh[k], std::true_type{});
        }
      }
      __syncwarp();
      flush_rows(flushed + 1, R);  // the rest of lane 31's high-half rows
      if constexpr (MODE == kModeLocal)
        best_abs = ::max(best_abs, ::max(lo16(best) + b[0], hi16(best) + b[1]));
      __syncwarp();
    }

    int v;
    if constexpr (MODE == kModeLocal) v = group_max<32>(best_abs);
    else if constexpr (MODE == kModeSemi) v = group_max<32>(rowmax);
    else v = gscore;
    if constexpr (MODE == kModeGlobal) {
      if (got) p.scores[pid] = v;
    } else if (t == 0) {
      p.scores[pid] = v;
    }
    __syncwarp();
  }
}

}  // namespace ga
