// ga_long.cuh -- multi-stage warp kernel for long pairs and for alphabets of
// more than four symbols (int32 cells).
//
// The columns (shorter sequence) are cut into stages of W = 32*K columns
// that one warp computes one after another from left to right, the
// multi-stage partitioning of a long alignment in Sec. 3.1.  A warp
// runs one pair: within a stage lane t owns K columns and works on row
// it - t + 1 as in the inter-sequence kernel; the right edge of a stage
// (H and the outgoing F of lane 31, one int2 per row) goes to a per-warp
// global buffer that lane 0 of the next stage reads.  Both directions are
// batched through shared memory every 32 rows with coalesced loads and
// stores, as the paper batches its boundary traffic every p iterations.
// One buffer serves all stages in place: a row is always read by the next
// stage's prefetch before the current stage's flush overwrites it.
//
// Substitution scores: for alphabets of <= 4 symbols the per-column
// byte-permute selectors of the inter-sequence kernel; otherwise a scoring
// profile of the stage in shared memory, P[c][x] = sigma(c, column x) as
// int8, one 16-byte load per 16 columns and a sign-extending prmt per
// column (Sec. 3.1, "scoring profile").
#pragma once

#include "ga_dp.cuh"

namespace ga {

struct KBParams {
  const uint32_t *packed_q;  // flat 2-bit codes (alphabets of <= 4), else unused
  const uint32_t *packed_t;
  const uint8_t *q_codes;    // raw codes (profile path)
  const uint8_t *t_codes;
  const int64_t *q_off;
  const int64_t *t_off;
  const int4 *info;
  const int32_t *sorted;
  const int32_t *range;
  int32_t *task_counter;
  uint32_t tables[16];       // table words as in KAParams
  int8_t sigma[32 * 32];     // A*A row-major sigma(query, target)
  int32_t A;
  int32_t alpha, beta;
  int32_t *scores;
  int2 *bnd;                 // per warp slot: bnd_stride int2 entries
  int64_t bnd_stride;
  int64_t nt, q0;            // cross chunk: pair p = (q0 + p/nt, p%nt); batch: nt = 0
};

template <int MODE, int K, bool PROFILE>
__global__ void __launch_bounds__(128) kb_kernel(const __grid_constant__ KBParams p) {
  using Cell = CellS32;
  using T = int32_t;
  constexpr int kWarps = 4;
  constexpr int W = 32 * K;
  constexpr int kNeg = kNeg32;
  static_assert(!PROFILE || (K % 16) == 0, "profile path loads 16 columns at a time");

  extern __shared__ __align__(16) uint8_t dyn_smem[];
  __shared__ int2 in_ring_s[kWarps][64];
  __shared__ int2 out_ring_s[kWarps][64];
  __shared__ uint32_t row_ring_s[kWarps][128];

  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  int2 *in_ring = in_ring_s[warp];
  int2 *out_ring = out_ring_s[warp];
  uint32_t *row_ring = row_ring_s[warp];
  uint8_t *prof = dyn_smem + (size_t)warp * (size_t)(p.A + 1) * W;  // PROFILE only
  int2 *bnd = p.bnd + (size_t)(blockIdx.x * kWarps + warp) * (size_t)p.bnd_stride;

  const int npairs = p.range[1] - p.range[0];
  const int alpha = p.alpha, beta = p.beta;
  const T NB = -beta;

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
    const int64_t rowpos = sw ? ts : qs;  // first residue in the flat packed stream
    const int64_t colpos = sw ? qs : ts;
    const uint32_t *rowbase = sw ? p.packed_t : p.packed_q;
    const uint32_t *colbase = sw ? p.packed_q : p.packed_t;
    const uint8_t *rowraw = sw ? p.t_codes + ts : p.q_codes + qs;
    const uint8_t *colraw = sw ? p.q_codes + qs : p.t_codes + ts;

    const int nst = (C + W - 1) / W;
    T best = 0;
    int rowmax = 0, gscore = 0;
    bool got = false;

    for (int s = 0; s < nst; ++s) {
      const int col0 = s * W;
      // ---- columns of this stage --------------------------------------
      T sel[PROFILE ? 1 : K];
      T na[MODE == kModeSemi ? K : 1];  // semi: column n frees its outgoing gaps
      T H[K], E[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int col = col0 + t * K + j;
        if constexpr (!PROFILE) {
          const int c = (col < C) ? packed_code(colbase, colpos + col) : -1;
          const uint32_t n0 = (c >= 0) ? (uint32_t)c : 8u;
          const uint32_t n1 = (c >= 0) ? (uint32_t)(c + 8) : 8u;
          sel[j] = (T)(n0 | (n1 << 4) | (n1 << 8) | (n1 << 12));
        }
        if constexpr (MODE == kModeSemi) na[j] = (col == C - 1) ? 0 : -alpha;
        H[j] = (MODE == kModeGlobal) ? ::max(-alpha - beta * col, kNeg) : 0;  // H(0, col+1)
        E[j] = ::max(H[j] - alpha, kNeg);  // E(1, col+1) = H(0, col+1) - alpha
      }
      if constexpr (PROFILE) {
        // P[c][x] = sigma(row residue c, column residue x); pad row c = A
        // and pad columns are 0.
        for (int e = t; e < (p.A + 1) * W; e += 32) {
          const int c = e / W, x = e - c * W;
          const int col = col0 + x;
          int v = 0;
          if (c < p.A && col < C) {
            const int cc = colraw[col];
            v = sw ? p.sigma[cc * p.A + c] : p.sigma[c * p.A + cc];
          }
          prof[e] = (uint8_t)(int8_t)v;
        }
      }
      const int ocol = C - 1 - col0 - t * K;  // local index of column n, if in this tile

      // ---- boundary of the stage's left edge --------------------------
      auto left_row = [&](int r) -> int2 {  // (H(r, col0), F(r, col0+1))
        int2 v;
        if (s == 0) {  // column 0: H(r, 0) and F(r, 1) = H(r, 0) - alpha
          v.x = (MODE == kModeGlobal) ? ((r == 0) ? 0 : ::max(-alpha - beta * (r - 1), kNeg)) : 0;
          v.y = ::max(v.x - alpha, kNeg);
        } else {
          v = in_ring[(r - 1) & 63];
        }
        return v;
      };
      auto load_batch = [&](int b) {  // rows 32b+1 .. 32b+32 -> in_ring
        if (s > 0) {
          const int r = 32 * b + 1 + t;
          in_ring[(r - 1) & 63] = bnd[r];
        }
      };
      auto fill_rows = [&](int b) {  // row table words / row codes, 4 batches
        const int r = 32 * b + 1 + t;
        uint32_t v;
        if (r > R) v = PROFILE ? (uint32_t)p.A : 0u;
        else if constexpr (PROFILE) v = rowraw[r - 1];
        else v = p.tables[(sw ? 8 : 0) + packed_code(rowbase, rowpos + r - 1)];
        row_ring[r & 127] = v;
      };
      load_batch(0);
      fill_rows(0);
      fill_rows(1);
      __syncwarp();

      const int h00 = (MODE == kModeGlobal && col0 > 0) ? ::max(-alpha - beta * (col0 - 1), kNeg) : 0;
      int hdt = 0;  // H(0, col0 + t*K)
      if constexpr (MODE == kModeGlobal) hdt = (col0 + t * K == 0) ? 0 : ::max(-alpha - beta * (col0 + t * K - 1), kNeg);
      const int2 l1 = left_row(1);
      T Hdiag = (t == 0) ? h00 : hdt;
      T Hleft = (t == 0) ? l1.x : hdt;
      T Fin = (t == 0) ? l1.y : kNeg;

      const int nit = R + 31;
      for (int it = 0; it < nit; ++it) {
        if ((it & 31) == 0) {
          __syncwarp();  // lane 31's out_ring rows are visible to the flush
          load_batch(it / 32 + 1);
          fill_rows(it / 32 + 2);
          if (it >= 64) {  // flush lane-31 rows (it-63 .. it-32)
            const int r = it - 63 + t;
            bnd[r] = out_ring[(r - 1) & 63];
          }
          __syncwarp();
        }
        const int r = it - t + 1;
        T Hout, Fout;
        if ((unsigned)(r - 1) < (unsigned)R) {
          const uint32_t rv = row_ring[r & 127];
          if constexpr (PROFILE) {
            const uint4 *pr = reinterpret_cast<const uint4 *>(prof + (size_t)rv * W + t * K);
            uint32_t w[K / 4];
#pragma unroll
            for (int q = 0; q < K / 16; ++q) {
              const uint4 v = pr[q];
              w[4 * q + 0] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
            }
            Fout = dp_row<Cell, MODE, K>(
                H, E, Hdiag, Fin, NB, best,
                [&](int j) -> T { return (T)prmt(w[j >> 2], 0u, sext_sel<Cell>(j & 3)); },
                [&](int j) -> T {
                  if constexpr (MODE == kModeSemi) return na[j];
                  else return -alpha;
                });
          } else {
            Fout = dp_row<Cell, MODE, K>(
                H, E, Hdiag, Fin, NB, best,
                [&](int j) -> T { return (T)prmt(rv, rv, (uint32_t)sel[j]); },
                [&](int j) -> T {
                  if constexpr (MODE == kModeSemi) return na[j];
                  else return -alpha;
                });
          }
          Hout = H[K - 1];
          if (r == R) {
            if constexpr (MODE == kModeGlobal) {
              if (ocol >= 0 && ocol < K) {
                T v = H[0];
#pragma unroll
                for (int j = 1; j < K; ++j)
                  if (j == ocol) v = H[j];
                gscore = v;
                got = true;
              }
            } else if constexpr (MODE == kModeSemi) {
#pragma unroll
              for (int j = 0; j < K; ++j) rowmax = ::max(rowmax, H[j]);
            }
          }
        } else {
          Hout = H[K - 1];
          Fout = kNeg;
        }
        if (t == 31 && r >= 1 && r <= R) out_ring[(r - 1) & 63] = make_int2(Hout, Fout);
        Hdiag = Hleft;
        Hleft = __shfl_up_sync(0xffffffffu, Hout, 1);
        Fin = __shfl_up_sync(0xffffffffu, Fout, 1);
        if (t == 0) {
          const int2 lv = (it + 2 <= R) ? left_row(it + 2) : make_int2(0, kNeg);
          Hleft = lv.x;
          Fin = lv.y;
        }
      }
      // flush the remaining lane-31 rows of this stage
      __syncwarp();
      {
        const int first = (nit >= 64) ? ((nit - 1) / 32) * 32 - 63 + 32 : 1;  // first unflushed row
        for (int r = first + t; r <= R; r += 32) bnd[r] = out_ring[(r - 1) & 63];
      }
      __syncwarp();
    }

    int v;
    if constexpr (MODE == kModeLocal) v = group_max<32>(best);
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
