// ga_bandpk.cuh -- packed int16x2 band-doubling kernel (global mode,
// alphabets of <= 4 symbols): the region, certificate and doubling of
// kc_kernel (ga_banded.cuh), with two adjacent stages of the pair in the two
// int16 halves of every register.
//
// Mapping.  A pair runs on a group of G lanes (G = 32: a warp; G = 16: two
// pairs per warp, neighbours in the band order, so alike in super-stages
// and window length, run in lockstep: the warp's loops run to the larger of
// the two, and a group past its own rows or pair runs with empty windows).
// A super-stage covers 2 x G x K columns: lane t of the group owns block
// col0 + tK (low halves) and block col0 + GK + tK (high halves).  The low
// half of lane t runs row r0 + it - t, where r0 is the first row of the low
// stage's region; the high half runs G rows behind, so that lane 0's high
// half receives lane G-1's low half one iteration after it produced the row
// (as in the packed long kernel, ga_longpk.cuh).  Every block runs only the
// rows of its window of the block-rounded band; a half outside its window
// computes values that nothing reads: its state is reset to the window's
// initial values when the window opens, its outputs are replaced by -inf by
// the receiving lane (the per-half select of kc_kernel), and the right edge
// (lane G-1's high half) is stored only inside the window.  A band's blocks
// enter their windows K + 1 iterations apart, so on a narrow band few of a
// super-stage's 2G blocks are inside at once; two super-stages of G = 16
// lanes side by side keep more lanes busy than one of 32.
//
// Relative int16 values with one base per half for the group.  The cells a
// half holds inside their windows at one iteration lie within G rows and GK
// columns of each other; adjacent cells differ by at most sigma_max +
// alpha, so with the bases renormalised every kKdRenorm iterations (to the H
// of a lane that is inside its window) every value in play stays within
// (sigma_max + alpha) * (2 * GK + 2G + kKdRenorm + 2) of its base, inside
// int16 when sigma_max + alpha <= kKdMaxStep.  -inf is kNeg16; a
// renormalisation saturates and re-clamps it, so that it stays below every
// real value.  Lane 0 converts the low half of lane G-1 into its high half
// with the base difference of the two halves, and the stage edges (global
// memory, batched through shared memory) hold absolute int32 values.
#pragma once

#include "ga_banded.cuh"
#include "ga_longpk.cuh"

namespace ga {

constexpr int kKdRenorm = 128;
// (2 * 32K + 2G + 128 + 2) * 24 = 29,232 < 32,000 - 2 * 24 at K = 16,
// G = 32 (16,128 at G = 16).
constexpr int kKdMaxStep = 24;

// Three resident blocks per SM: without the bound ptxas takes 255 registers
// (one block) for the two row-step variants.
template <int K, int G>
__global__ void __launch_bounds__(128, 3) kd_kernel(const __grid_constant__ KCParams p) {
  static_assert(G == 16 || G == 32, "lanes per pair");
  constexpr int kWarps = 4;
  constexpr int kGroups = 32 / G;       // pairs per warp, one per group of G lanes
  constexpr int kRowsPerLane = 32 / G;  // rows of a 32-row batch per lane
  constexpr int W = G * K;    // columns per half (one kc_kernel stage when G = 32)
  constexpr int W2 = 2 * W;   // columns per super-stage
  constexpr int kRing = 256;  // row table words by row & 255
  constexpr int kNeg = kNeg32;

  __shared__ int2 in_ring_s[kWarps * kGroups][64];
  __shared__ int2 out_ring_s[kWarps * kGroups][64];
  __shared__ uint32_t row_ring_s[kWarps * kGroups][kRing + 32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / G, t = lane % G, gl0 = g * G;  // group, lane in the group, its first lane
  const unsigned glow = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
  const int left_lane = gl0 + (t + G - 1) % G;  // the lane of the group's previous block
  int2 *in_ring = in_ring_s[warp * kGroups + g];
  int2 *out_ring = out_ring_s[warp * kGroups + g];
  uint32_t *row_ring = row_ring_s[warp * kGroups + g];
  int2 *bnd = p.bnd + ((size_t)(blockIdx.x * kWarps + warp) * kGroups + g) * (size_t)p.bnd_stride;
  const int alpha = p.alpha, beta = p.beta;
  const uint32_t NB = pk16(-beta, -beta);
  const uint32_t NAc = pk16(-alpha, -alpha);
  const uint32_t NEGV = pk16(kNeg16, kNeg16);

  const int npairs = p.range[1] - p.range[0];
  for (;;) {
    // ---- a task: kGroups consecutive pairs of the order, one per group;
    // the groups run in lockstep (warp-wide loop bounds), a group whose pair
    // is done (or that has none) runs with empty windows -----------------
    int task = 0;
    if (lane == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task * kGroups >= npairs) break;
    const int idx = task * kGroups + g;
    bool done = idx >= npairs;
    const int pid = done ? 0 : p.order[p.range[0] + idx];
    const int64_t qs = done ? 0 : p.q_off[pid], ts = done ? 0 : p.t_off[pid];
    int m = done ? 0 : (int)(p.q_off[pid + 1] - qs), n = done ? 0 : (int)(p.t_off[pid + 1] - ts);
    const bool bisect = p.bis_lo != nullptr;
    int w = 0;
    if (!done) {
      if (bisect) {
        const int lw = p.bis_lo[pid], hw = p.bis_hi[pid];
        if (lw >= hw) done = true;
        w = lw + (hw - lw) / 2;
      } else {
        w = p.w0 ? p.w0[pid] : p.default_w0;
      }
    }
    if (w < 0) w = 0;
    if (!done && (m == 0 || n == 0)) {  // closed form, any band
      if (t == 0) {
        if (bisect) {
          p.bis_lo[pid] = p.bis_hi[pid] = 0;
        } else {
          const int len = m + n;
          p.scores[pid] = len ? -(alpha + beta * (len - 1)) : 0;
          if (p.w_used) p.w_used[pid] = w;
        }
      }
      done = true;
    }
    if (done) m = n = 0;
    const int dn = n - m;
    unsigned long long tries = 0, cells = 0;

    for (;;) {  // one attempt of every group's pair per round
      if (!__any_sync(0xffffffffu, !done)) break;
      const int lo = (dn < 0 ? dn : 0) - w;
      const int hi = (dn > 0 ? dn : 0) + w;
      const int nst2 = done ? 0 : (n + W2 - 1) / W2;
      const int nst2w = (int)__reduce_max_sync(0xffffffffu, (unsigned)nst2);
      int S = kNeg;
      for (int s2 = 0; s2 < nst2w; ++s2) {
        const bool sact = s2 < nst2;  // this group has a super-stage s2
        const int col0 = s2 * W2;
        // ---- blocks and windows of both halves --------------------------
        int cb[2], wlo[2], whi[2], plo[2], phi[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cb[h] = col0 + h * W + t * K;
          wlo[h] = ::max(1, cb[h] + 1 - hi);
          whi[h] = ::min(m, cb[h] + K - lo);
          const int pb = cb[h] - K;
          plo[h] = (cb[h] == 0) ? 0 : ::max(1, pb + 1 - hi);
          phi[h] = (cb[h] == 0) ? ::min(m, -lo) : ::min(m, pb + K - lo);
          if (!sact) {  // no super-stage s2 for this group: empty windows
            wlo[h] = plo[h] = 1;
            whi[h] = phi[h] = 0;
          }
          if (wlo[h] <= whi[h] && cb[h] < n)
            cells += (unsigned long long)(whi[h] - wlo[h] + 1) * (unsigned long long)::min(K, n - cb[h]);
        }
        // first row of the low stage (lane 0's window), last row of the last
        // real block, iterations of this group and of the warp
        const int r0 = sact ? ::max(1, col0 + 1 - hi) : 1;
        const int cend = ::min(col0 + W2, n);     // real columns of the super-stage
        const int cbl = ((cend - 1) / K) * K;     // last real block
        const int r_end = sact ? ::min(m, cbl + K - lo) : 0;
        const bool high_real = sact && cend > col0 + W;
        const int nit_g = sact ? ::max(0, (r_end - r0 + 1) + (high_real ? 2 * G - 1 : G - 1)) : 0;
        const int nit = (int)__reduce_max_sync(0xffffffffu, (unsigned)nit_g);
        const bool edge_out = sact && s2 + 1 < nst2;  // the next super-stage reads this one's edge
        // the owner of column n (0-based n-1) and its half
        const int oc = n - 1 - col0;
        const bool own_stage = oc < W2;
        const int oh = oc >= W ? 1 : 0;
        const bool owner = sact && own_stage && t == (oc - oh * W) / K;
        const int oj = (oc - oh * W) % K;

        uint32_t sel[K], H[K], E[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          uint32_t sv = 0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int col = cb[h] + j;
            const int c = (col < n) ? packed_code(p.packed_t, ts + col) : -1;
            const uint32_t n0 = (c >= 0) ? (uint32_t)(c + 4 * h) : (uint32_t)(8 + 4 * h);
            const uint32_t n1 = (c >= 0) ? (uint32_t)(c + 4 * h + 8) : (uint32_t)(8 + 4 * h);
            sv |= (n0 | (n1 << 4)) << (8 * h);
          }
          sel[j] = sv;
          H[j] = NEGV;  // set when each half's window opens
          E[j] = NEGV;
        }
        // bases: the low half's from the left edge of its first row, the
        // high half's the same until it has a lane inside its window
        int b0 = 0;  // super-stage 0 starts at row 1 next to H(0, 0) = 0
        if (sact && s2 > 0 && t == 0) b0 = bnd[::min(r0, phi[0])].x;  // a row of the left edge near row r0
        b0 = __shfl_sync(0xffffffffu, b0, gl0);
        int b1 = b0;

        auto col0_h = [&](int r) -> int {  // column 0, strict band rule (absolute)
          return (r <= -lo) ? (r == 0 ? 0 : -alpha - beta * (r - 1)) : kNeg;
        };
        auto row0_h = [&](int c) -> int {  // H(0, c), absolute, for 1-based column c >= 1
          return -alpha - beta * (c - 1);
        };
        // rows of batch bb: r0 + 32bb .. r0 + 32bb + 31, kRowsPerLane per lane;
        // the warp may run past this group's rows (another group's longer
        // stage), so only rows up to m are read
        auto load_batch = [&](int bb) {
          if (s2 > 0) {
#pragma unroll
            for (int k = 0; k < kRowsPerLane; ++k) {
              const int r = r0 + 32 * bb + t + G * k;
              if (r <= m) in_ring[(r - r0) & 63] = bnd[r];
            }
          }
        };
        auto fill_rows = [&](int bb) {
#pragma unroll
          for (int k = 0; k < kRowsPerLane; ++k) {
            const int r = r0 + 32 * bb + t + G * k;
            uint32_t v = 0;
            if (r <= m) v = p.tables[packed_code(p.packed_q, qs + r - 1)];
            const int x = r & (kRing - 1);
            row_ring[x] = v;
            if (x < 32) row_ring[x + kRing] = v;  // mirror: a batch's rows are contiguous
          }
        };
        // lane 0's low-half left input (H(r, col0), F(r, col0 + 1)) relative
        // to base b, -inf outside the left block's window
        auto lane0_left = [&](int r, int b, int &hl, int &fl) {
          if (r < plo[0] || r > phi[0] || r < 1) {
            hl = kNeg16;
            fl = kNeg16;
          } else if (s2 == 0) {
            const int hv = col0_h(r);
            hl = (hv == kNeg) ? kNeg16 : hv - b;
            fl = (hv == kNeg) ? kNeg16 : hv - alpha - b;
          } else {
            const int2 v = in_ring[(r - r0) & 63];
            hl = v.x - b;
            fl = v.y - b;
          }
        };
        load_batch(0);
        fill_rows(0);
        fill_rows(1);
        __syncwarp();

        uint32_t Hdiag = NEGV, Hleft = NEGV, Fin = NEGV;
        // One row step with the per-row window logic.
        auto step_general = [&](int it) {
          const int rl = r0 + it - t, rh = rl - G;
          // a half's window opens: its state becomes the window's row wlo - 1
          if (rl == wlo[0] || rh == wlo[1]) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if ((h ? rh : rl) != wlo[h]) continue;
              const int b = h ? b1 : b0;
              const uint32_t keep = h ? 0x0000ffffu : 0xffff0000u;
#pragma unroll
              for (int j = 0; j < K; ++j) {
                int hv = kNeg16, ev = kNeg16;
                if (wlo[h] == 1) {  // row 0 of the block
                  hv = row0_h(cb[h] + j + 1) - b;
                  ev = hv - alpha;
                }
                H[j] = (H[j] & keep) | (pk16(hv, hv) & ~keep);
                E[j] = (E[j] & keep) | (pk16(ev, ev) & ~keep);
              }
              int hd = kNeg16;  // H(wlo - 1, cb): the left block's last column
              bool set_diag = false;
              if (t == 0 && h == 0) {
                set_diag = true;
                if (wlo[0] - 1 == 0) {
                  hd = (cb[0] == 0) ? -b : ((plo[0] == 1) ? row0_h(cb[0]) - b : kNeg16);
                } else if (wlo[0] - 1 < plo[0] || wlo[0] - 1 > phi[0]) {
                  hd = kNeg16;
                } else if (s2 == 0) {
                  const int hv = col0_h(wlo[0] - 1);
                  hd = (hv == kNeg) ? kNeg16 : hv - b;
                } else {
                  hd = bnd[wlo[0] - 1].x - b;
                }
                int hl, fl;
                lane0_left(wlo[0], b, hl, fl);
                Hleft = (Hleft & keep) | (pk16(hl, hl) & ~keep);
                Fin = (Fin & keep) | (pk16(fl, fl) & ~keep);
              } else if (wlo[h] - 1 == 0) {
                set_diag = true;
                hd = (plo[h] == 1) ? row0_h(cb[h]) - b : kNeg16;
              }
              if (set_diag) Hdiag = (Hdiag & keep) | (pk16(hd, hd) & ~keep);
            }
          }
          const bool in0 = rl >= wlo[0] && rl <= whi[0];
          const bool in1 = rh >= wlo[1] && rh <= whi[1];
          uint32_t Hout = NEGV, Fout = NEGV;
          if (in0 || in1) {
            const uint32_t twl = row_ring[rl & (kRing - 1)];
            const uint32_t twh = row_ring[rh & (kRing - 1)];
            uint32_t unused_best = 0;
            Fout = pk_row<kModeGlobal, K>(
                H, E, Hdiag, Fin, NB, 0u, unused_best, [&](int j) -> uint32_t { return prmt(twl, twh, sel[j]); },
                [&](int) -> uint32_t { return NAc; });
            Hout = H[K - 1];
            if (owner && (oh ? (rh == m && in1) : (rl == m && in0))) {
              uint32_t v = H[0];
#pragma unroll
              for (int j = 1; j < K; ++j)
                if (j == oj) v = H[j];
              S = oh ? hi16(v) + b1 : lo16(v) + b0;
            }
          }
          if (t == G - 1 && in1) out_ring[(rh - r0) & 63] = make_int2(hi16(Hout) + b1, hi16(Fout) + b1);
          // next row's inputs: lane t-1's outputs, -inf outside its window;
          // lane 0: the edge (low half) and lane 31's low half (high half)
          const int rn0 = rl + 1, rn1 = rh + 1;
          uint32_t hs = __shfl_sync(0xffffffffu, Hout, left_lane);
          uint32_t fs = __shfl_sync(0xffffffffu, Fout, left_lane);
          if (t == 0) {
            int hl, fl;
            lane0_left(rn0, b0, hl, fl);
            const uint32_t dlh = pk16(0, b0 - b1);
            hs = __vadd2(prmt((uint32_t)hl, hs, 0x5410u), dlh);
            fs = __vadd2(prmt((uint32_t)fl, fs, 0x5410u), dlh);
          }
          const bool ok0 = (t == 0) || (rn0 >= plo[0] && rn0 <= phi[0]);
          const bool ok1 = rn1 >= plo[1] && rn1 <= phi[1];
          const uint32_t okm = (ok0 ? 0x0000ffffu : 0u) | (ok1 ? 0xffff0000u : 0u);
          Hdiag = Hleft;
          Hleft = (hs & okm) | (NEGV & ~okm);
          Fin = (fs & okm) | (NEGV & ~okm);
        };
        // One row step of an iteration in which every lane is strictly inside
        // both of its windows, every input from its left neighbour lies inside
        // that neighbour's window and no lane is at row m: the same step
        // without the window logic.
        auto step_fast = [&](int it, uint32_t twl, uint32_t twh) {
          const int rl = r0 + it - t;
          int hl = kNeg16, fl = kNeg16;
          if (t == 0) lane0_left(rl + 1, b0, hl, fl);  // read before the row update
          uint32_t unused_best = 0;
          const uint32_t Fout = pk_row<kModeGlobal, K>(
              H, E, Hdiag, Fin, NB, 0u, unused_best, [&](int j) -> uint32_t { return prmt(twl, twh, sel[j]); },
              [&](int) -> uint32_t { return NAc; });
          const uint32_t Hout = H[K - 1];
          if (t == G - 1) out_ring[(rl - G - r0) & 63] = make_int2(hi16(Hout) + b1, hi16(Fout) + b1);
          uint32_t hs = __shfl_sync(0xffffffffu, Hout, left_lane);
          uint32_t fs = __shfl_sync(0xffffffffu, Fout, left_lane);
          if (t == 0) {
            const uint32_t dlh = pk16(0, b0 - b1);
            hs = __vadd2(prmt((uint32_t)hl, hs, 0x5410u), dlh);
            fs = __vadd2(prmt((uint32_t)fl, fs, 0x5410u), dlh);
          }
          Hdiag = Hleft;
          Hleft = hs;
          Fin = fs;
        };
        // the iterations [fa, fb] where step_fast applies to every lane
        int fa, fb;
        {
          int a = ::max(wlo[0] + 1, wlo[1] + G + 1) - r0 + t;
          int z = ::min(::min(whi[0], m - 1), ::min(whi[1], m - 1) + G) - r0 + t;
          a = ::max(a, plo[1] + G - 1 - r0 + t);  // high-half input rows rh + 1
          z = ::min(z, phi[1] + G - 1 - r0 + t);
          if (t > 0) {  // low-half input rows rl + 1 (lane 0 checks its edge itself)
            a = ::max(a, plo[0] - 1 - r0 + t);
            z = ::min(z, phi[0] - 1 - r0 + t);
          }
          if (!sact) {  // a group without this super-stage constrains nothing
            a = -(1 << 29);
            z = 1 << 29;
          }
          fa = __reduce_max_sync(0xffffffffu, a);
          fb = __reduce_min_sync(0xffffffffu, z);
        }
        // lane G-1's high-half edge rows r0 .. flushed are in bnd; a batch
        // flushes the rows stored since the last one (at most 32)
        int flushed = r0 - 1;
        for (int it0 = 0; it0 < nit; it0 += 32) {
          __syncwarp();
          load_batch(it0 / 32 + 1);
          fill_rows(it0 / 32 + 2);
          if (edge_out) {  // the last stored row: r0 + it0 - 2G (iteration it0 - 1)
            const int last = ::min(r0 + it0 - 2 * G, r_end);
#pragma unroll
            for (int k = 0; k < kRowsPerLane; ++k) {
              const int r = flushed + 1 + t + G * k;
              if (r <= last) bnd[r] = out_ring[(r - r0) & 63];
            }
            flushed = ::max(flushed, last);
          }
          if ((it0 & (kKdRenorm - 1)) == 0 && it0 > 0) {
            // each half's base moves to the H of its first lane whose state
            // (the row before its current one) lies inside its window; a
            // half with no such lane follows the other half
            const int rl = r0 + it0 - t - 1, rh = rl - G;
            const unsigned in0 = (__ballot_sync(0xffffffffu, rl >= wlo[0] && rl <= whi[0]) >> gl0) & glow;
            const unsigned in1 = (__ballot_sync(0xffffffffu, rh >= wlo[1] && rh <= whi[1]) >> gl0) & glow;
            const uint32_t h0v = __shfl_sync(0xffffffffu, H[0], gl0 + (in0 ? __ffs(in0) - 1 : 0));
            const uint32_t h1v = __shfl_sync(0xffffffffu, H[0], gl0 + (in1 ? __ffs(in1) - 1 : 0));
            int d0 = in0 ? lo16(h0v) : 0;
            int d1 = in1 ? hi16(h1v) : 0;
            if (!in0 && in1) d0 = b1 + d1 - b0;
            if (!in1) d1 = b0 + d0 - b1;
            b0 += d0;
            b1 += d1;
            const uint32_t dl = pk16(d0, d1);
#pragma unroll
            for (int j = 0; j < K; ++j) {
              H[j] = __vmaxs2(__vsubss2(H[j], dl), NEGV);
              E[j] = __vmaxs2(__vsubss2(E[j], dl), NEGV);
            }
            Hdiag = __vmaxs2(__vsubss2(Hdiag, dl), NEGV);
            Hleft = __vmaxs2(__vsubss2(Hleft, dl), NEGV);
            Fin = __vmaxs2(__vsubss2(Fin, dl), NEGV);
          }
          __syncwarp();
          if (it0 >= fa && it0 + 31 <= fb) {
            // this lane's ring entries of the batch are contiguous (mirrored ring)
            const uint32_t *rpl = row_ring + ((r0 + it0 - t) & (kRing - 1));
            const uint32_t *rph = row_ring + ((r0 + it0 - t - G) & (kRing - 1));
#pragma unroll 2
            for (int k = 0; k < 32; ++k) step_fast(it0 + k, rpl[k], rph[k]);
          } else {
            const int nb = ::min(32, nit - it0);
#pragma unroll 1
            for (int k = 0; k < nb; ++k) step_general(it0 + k);
          }
        }
        __syncwarp();
        if (edge_out) {  // the rest of lane G-1's high-half rows
          for (int r = flushed + 1 + t; r <= r_end; r += G) bnd[r] = out_ring[(r - r0) & 63];
        }
        __syncwarp();
      }
      // certificate (as kc_kernel), per group
      S = group_max<G>(S);
      if (!done) {
        const bool covers = (lo <= -m) && (hi >= n);
        int64_t ub = INT64_MIN;
        if (lo - 1 >= -m) ub = ::max(ub, band_ub(m, n, p.sigma_max_pos, alpha, beta, lo - 1));
        if (hi + 1 <= n) ub = ::max(ub, band_ub(m, n, p.sigma_max_pos, alpha, beta, hi + 1));
        if (bisect) {
          if (t == 0) {
            if (covers || (int64_t)S >= ub) p.bis_hi[pid] = w;
            else p.bis_lo[pid] = w + 1;
          }
          done = true;
        } else if (covers || (int64_t)S >= ub) {
          if (t == 0) {
            p.scores[pid] = S;
            if (p.w_used) p.w_used[pid] = w;
          }
          done = true;
        } else {
          w = (w == 0) ? 1 : 2 * w;
          ++tries;
        }
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cells += __shfl_xor_sync(0xffffffffu, cells, o);
    if (t == 0 && tries) atomicAdd(p.retries, tries);
    if (lane == 0) atomicAdd(p.cells, cells);
  }
}

}  // namespace ga
