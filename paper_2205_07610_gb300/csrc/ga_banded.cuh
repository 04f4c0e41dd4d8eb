// ga_banded.cuh -- global alignment restricted to a band of diagonals, with
// the band-doubling certificate (not part of the paper; the classic
// Ukkonen / Fickett argument).
//
// Region.  For w the band is [lo, hi] = [min(0,n-m) - w, max(0,n-m) + w]
// (d = j - i).  The kernel computes the band rounded out to blocks of K = 16
// columns: block b (columns bK+1 .. bK+K) runs rows max(1, bK+1-hi) ..
// min(m, bK+K-lo), its row-0 cells belong to the region when that range
// starts at row 1, and column-0 cells when -i >= lo.  Every cell outside the
// region is -inf.  The region contains the band, so a path that leaves the
// computed region visits a diagonal outside [lo, hi] and is bounded by
//     UB(d) = max(sigma_max,0) * (m+n-g)/2 - (alpha*r + beta*(g-r)),
//     g = |d| + |d-(n-m)|,  r = 2 outside [min(0,n-m), max(0,n-m)], else (g > 0).
// The region score S is accepted when S >= UB of the nearest diagonals
// outside the band (a band covering the matrix is always accepted); else w
// doubles.  The accepted S equals the full-DP score.
//
// Mapping: one warp per pair, 32 lanes x K columns per stage (Sec. 3.1
// multi-stage partitioning), exactly as the long-pair kernel, but each lane
// only runs the rows of its block's window and every value received from a
// neighbour outside its window is replaced by -inf; a stage only iterates
// the rows where any of its blocks is inside the band.  The stage edge goes
// through a per-warp global buffer batched in shared memory.
#pragma once

#include "ga_dp.cuh"

namespace ga {

struct KCParams {
  const uint32_t *packed_q;  // flat 2-bit codes
  const uint32_t *packed_t;
  const int64_t *q_off;
  const int64_t *t_off;
  const int32_t *order;      // pair ids, longest estimated work first
  const int32_t *range;      // [start, end) of the pairs to run in `order`
  int32_t *task_counter;
  uint32_t tables[16];
  int32_t alpha, beta;
  int32_t sigma_max_pos;
  const int32_t *w0;         // per pair, or nullptr
  int32_t default_w0;
  int32_t *scores;
  int32_t *w_used;           // nullable
  unsigned long long *retries;
  unsigned long long *cells;
  int2 *bnd;
  int64_t bnd_stride;
  // Bisection mode (both non-null): one attempt per pair at w = (lo+hi)/2 of
  // the pair's interval [lo, hi] of candidate minimal widths, which the
  // attempt then halves (certified: hi = w, else lo = w + 1); pairs with
  // lo == hi are skipped and nothing else is written.
  int32_t *bis_lo;
  int32_t *bis_hi;
};

__device__ __forceinline__ int64_t band_ub(int64_t m, int64_t n, int64_t smax, int64_t alpha,
                                           int64_t beta, int64_t d) {
  const int64_t dn = n - m;
  const int64_t lo_main = dn < 0 ? dn : 0, hi_main = dn > 0 ? dn : 0;
  const int64_t g = (d < 0 ? -d : d) + (d - dn < 0 ? dn - d : d - dn);
  const int64_t r = (d < lo_main || d > hi_main) ? 2 : (g > 0 ? 1 : 0);
  return smax * ((m + n - g) / 2) - (alpha * r + beta * (g - r));
}

template <int K>
__global__ void __launch_bounds__(128) kc_kernel(const __grid_constant__ KCParams p) {
  using Cell = CellS32;
  using T = int32_t;
  constexpr int kWarps = 4;
  constexpr int W = 32 * K;
  constexpr int kNeg = kNeg32;

  __shared__ int2 in_ring_s[kWarps][64];
  __shared__ int2 out_ring_s[kWarps][64];
  __shared__ uint32_t row_ring_s[kWarps][128];

  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  int2 *in_ring = in_ring_s[warp];
  int2 *out_ring = out_ring_s[warp];
  uint32_t *row_ring = row_ring_s[warp];
  int2 *bnd = p.bnd + (size_t)(blockIdx.x * kWarps + warp) * (size_t)p.bnd_stride;
  const int alpha = p.alpha, beta = p.beta;
  const T NB = -beta;
  const T NAc = -alpha;

  for (;;) {
    int task = 0;
    if (t == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= p.range[1] - p.range[0]) break;
    const int pid = p.order[p.range[0] + task];
    const int64_t qs = p.q_off[pid], ts = p.t_off[pid];
    const int m = (int)(p.q_off[pid + 1] - qs), n = (int)(p.t_off[pid + 1] - ts);
    const bool bisect = p.bis_lo != nullptr;
    int w;
    if (bisect) {
      const int lw = p.bis_lo[pid], hw = p.bis_hi[pid];
      if (lw >= hw) continue;
      w = lw + (hw - lw) / 2;
    } else {
      w = p.w0 ? p.w0[pid] : p.default_w0;
    }
    if (w < 0) w = 0;
    if (m == 0 || n == 0) {  // closed form, any band
      if (bisect) {  // w = 0 already covers the matrix
        if (t == 0) p.bis_lo[pid] = p.bis_hi[pid] = 0;
        continue;
      }
      if (t == 0) {
        const int len = m + n;
        p.scores[pid] = len ? -(alpha + beta * (len - 1)) : 0;
        if (p.w_used) p.w_used[pid] = w;
      }
      continue;
    }
    const int dn = n - m;
    const int nst = (n + W - 1) / W;
    unsigned long long tries = 0, cells = 0;

    for (;;) {
      const int lo = (dn < 0 ? dn : 0) - w;
      const int hi = (dn > 0 ? dn : 0) + w;
      int S = kNeg;
      for (int s = 0; s < nst; ++s) {
        const int col0 = s * W;  // 0-based first column of the stage
        const int cb = col0 + t * K;  // 0-based first column of this lane's block
        const int wlo = ::max(1, cb + 1 - hi), whi = ::min(m, cb + K - lo);
        // left neighbour's block window (lane t-1, or the previous stage's
        // last lane, or column 0)
        const int pb = cb - K;
        const int plo = (cb == 0) ? 0 : ::max(1, pb + 1 - hi);
        const int phi = (cb == 0) ? ::min(m, -lo) : ::min(m, pb + K - lo);
        const int r_lo = ::max(1, col0 + 1 - hi), r_hi = ::min(m, col0 + W - lo);
        if (wlo <= whi && cb < n)
          cells += (unsigned long long)(whi - wlo + 1) * (unsigned long long)::min(K, n - cb);
        // ---- columns of the block, row (wlo - 1) ----
        T sel[K], H[K], E[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int col = cb + j;
          const int c = (col < n) ? packed_code(p.packed_t, ts + col) : -1;
          const uint32_t n0 = (c >= 0) ? (uint32_t)c : 8u;
          const uint32_t n1 = (c >= 0) ? (uint32_t)(c + 8) : 8u;
          sel[j] = (T)(n0 | (n1 << 4) | (n1 << 8) | (n1 << 12));
          const int h0 = (wlo == 1) ? ::max(-alpha - beta * col, kNeg) : kNeg;  // H(0, col+1)
          H[j] = h0;
          E[j] = (h0 == kNeg) ? kNeg : ::max(h0 - alpha, kNeg);
        }
        const int ocol = n - 1 - cb;  // local index of column n, if in this block
        // value the left neighbour holds for row r (H(r, cb)), -inf outside
        auto left_h_row0 = [&]() -> int {  // H(0, cb): row-0 cell of the left block
          if (cb == 0) return 0;
          return (plo == 1) ? ::max(-alpha - beta * (cb - 1), kNeg) : kNeg;
        };
        auto col0_h = [&](int r) -> int {  // column 0, strict band rule
          return (r <= -lo) ? (r == 0 ? 0 : ::max(-alpha - beta * (r - 1), kNeg)) : kNeg;
        };
        // stage edge from the previous stage, batched (rows r_lo + 32b ..)
        auto load_batch = [&](int b) {
          if (s > 0) {
            const int r = r_lo + 32 * b + t;
            in_ring[(r - r_lo) & 63] = bnd[r];
          }
        };
        auto fill_rows = [&](int b) {
          const int r = r_lo + 32 * b + t;
          uint32_t v = 0;
          if (r <= m) v = p.tables[packed_code(p.packed_q, qs + r - 1)];
          row_ring[(r - r_lo) & 127] = v;
        };
        auto lane0_left = [&](int r, int &hl, int &fl) {  // lane 0's inputs for row r
          if (r < plo || r > phi || r < 1) {
            hl = kNeg;
            fl = kNeg;
          } else if (s == 0) {
            hl = col0_h(r);
            fl = (hl == kNeg) ? kNeg : hl - alpha;
          } else {
            const int2 v = in_ring[(r - r_lo) & 63];
            hl = v.x;
            fl = v.y;
          }
        };
        load_batch(0);
        fill_rows(0);
        fill_rows(1);
        __syncwarp();

        // diagonal and left inputs for row wlo of every lane are set when the
        // lane starts; lane 0 also receives through lane0_left.
        T Hdiag = kNeg, Hleft = kNeg, Fin = kNeg;
        const int nit = (r_hi - r_lo + 1) + 31;
        for (int it = 0; it < nit; ++it) {
          if ((it & 31) == 0) {
            __syncwarp();
            load_batch(it / 32 + 1);
            fill_rows(it / 32 + 2);
            if (it >= 64) {  // flush lane-31 rows r_lo + it - 64 .. r_lo + it - 33
              const int r = r_lo + it - 64 + t;
              bnd[r] = out_ring[(r - r_lo) & 63];
            }
            __syncwarp();
          }
          const int r = r_lo + it - t;
          // first row of this lane's window: diagonal is the left block's
          // row wlo-1 (a row-0 cell or an ordinary cell), left is row wlo
          if (r == wlo) {
            if (t == 0) {
              // row wlo - 1 = r_lo - 1 precedes the first staged batch
              int hd, hl, fl;
              if (wlo - 1 == 0) hd = left_h_row0();
              else if (wlo - 1 < plo || wlo - 1 > phi) hd = kNeg;
              else if (s == 0) hd = col0_h(wlo - 1);
              else hd = bnd[wlo - 1].x;
              lane0_left(wlo, hl, fl);
              Hdiag = hd;
              Hleft = hl;
              Fin = fl;
            } else if (wlo - 1 == 0) {
              Hdiag = left_h_row0();
            }
          }
          T Hout = kNeg, Fout = kNeg;
          if (r >= wlo && r <= whi) {
            const uint32_t rv = row_ring[(r - r_lo) & 127];
            T unused_best = 0;
            Fout = dp_row<Cell, kModeGlobal, K>(
                H, E, Hdiag, Fin, NB, unused_best,
                [&](int j) -> T { return (T)prmt(rv, rv, (uint32_t)sel[j]); },
                [&](int) -> T { return NAc; });
            Hout = H[K - 1];
            if (r == m && ocol >= 0 && ocol < K) {
              T v = H[0];
#pragma unroll
              for (int j = 1; j < K; ++j)
                if (j == ocol) v = H[j];
              S = v;
            }
          }
          if (t == 31 && r >= wlo && r <= whi) out_ring[(r - r_lo) & 63] = make_int2(Hout, Fout);
          // next row's inputs: shuffled from lane t-1, -inf outside its window
          const int rn = r + 1;
          const T hs = __shfl_up_sync(0xffffffffu, Hout, 1);
          const T fs = __shfl_up_sync(0xffffffffu, Fout, 1);
          if (t == 0) {
            int hl, fl;
            lane0_left(rn, hl, fl);
            Hdiag = Hleft;
            Hleft = hl;
            Fin = fl;
          } else {
            const bool ok = rn >= plo && rn <= phi;
            Hdiag = Hleft;
            Hleft = ok ? hs : kNeg;
            Fin = ok ? fs : kNeg;
          }
        }
        __syncwarp();
        {  // flush the remaining lane-31 rows of the stage
          const int done = (nit - 1 >= 64) ? ((nit - 1) / 32) * 32 - 32 : 0;  // rows r_lo .. r_lo+done-1 flushed
          for (int r = r_lo + done + t; r <= r_hi; r += 32) bnd[r] = out_ring[(r - r_lo) & 63];
        }
        __syncwarp();
      }
      // certificate
      S = __reduce_max_sync(0xffffffffu, S);  // only the owner lane holds H(m,n)
      const bool covers = (lo <= -m) && (hi >= n);
      int64_t ub = INT64_MIN;
      if (lo - 1 >= -m) ub = ::max(ub, band_ub(m, n, p.sigma_max_pos, alpha, beta, lo - 1));
      if (hi + 1 <= n) ub = ::max(ub, band_ub(m, n, p.sigma_max_pos, alpha, beta, hi + 1));
      if (bisect) {
        if (t == 0) {
          if (covers || (int64_t)S >= ub) p.bis_hi[pid] = w;
          else p.bis_lo[pid] = w + 1;
        }
        break;
      }
      if (covers || (int64_t)S >= ub) {
        if (t == 0) {
          p.scores[pid] = S;
          if (p.w_used) p.w_used[pid] = w;
        }
        break;
      }
      w = (w == 0) ? 1 : 2 * w;
      ++tries;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cells += __shfl_xor_sync(0xffffffffu, cells, o);
    if (t == 0) {
      if (tries) atomicAdd(p.retries, tries);
      atomicAdd(p.cells, cells);
    }
  }
}

}  // namespace ga
