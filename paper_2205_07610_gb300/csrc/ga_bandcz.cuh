// ga_bandcz.cuh -- packed int16x2 band-doubling kernel with a continuous
// block schedule (global mode, alphabets of <= 4 symbols): the region,
// certificate and doubling of kc_kernel (ga_banded.cuh), one pair per warp.
//
// Why a continuous schedule.  The region is the band rounded out to blocks of
// K = 16 target columns; block b runs the rows of its window [wlo_b, whi_b],
// B = hi - lo + K rows long, and each window starts K rows after its left
// neighbour's.  A warp holds 64 blocks at once (lane t owns one block in the
// low int16 halves of its registers and the block 32 further right in the
// high halves: 64 "lane-halves").  Run one super-stage of 64 blocks at a time
// and the super-stage lasts B + 17 * 63 iterations while each block is busy
// for B of them.  Here every lane-half moves on to its block of the next
// super-stage (64 blocks further right) as soon as its window closes:
// lane-half l runs row r of super-stage s at iteration r + l + T_s with
// T_s = D * s - 1, so a lane-half is busy B of every 1024 + D iterations.
//
// Spacing D = max(128, min(m, B - 63K) + 1):
//   * a window holds at most min(m, B) rows, so a lane-half's windows of
//     consecutive super-stages lie apart in time;
//   * a lane-half's left neighbour opens its next window only after the
//     lane-half's last row, so a lane-half that is outside its window (idle)
//     can send -inf to its right neighbour, every value a lane-half receives
//     inside its window is correct without a mask of its own, and a value a
//     neighbour sends from its new window reaches an idle lane-half
//     unconverted;
//   * D >= 127 puts the edge between super-stages (lane-half 63 of super-
//     stage s -> lane-half 0 of s + 1, D - 63 iterations later) through a
//     per-warp global FIFO that is loaded a batch of 32 iterations ahead.
//
// Relative int16 values with one base per lane-half.  Lane-halves of one
// warp can be in two super-stages 1024 + D iterations apart, so one base per
// half for the whole warp would not bound the values; each lane-half keeps
// its own int32 base instead.  A lane-half adopts its left
// neighbour's base when its window opens (lane-half 0: a value of the edge
// FIFO) and moves it to its own H every 128 iterations; the sender converts
// what it sends to the receiver's base (both inside their windows: the same
// super-stage, close bases) or sends it unconverted (receiver idle: the
// receiver adopts the sender's base when it opens).  Every value a lane-half
// holds inside its window stays within (sigma_max + alpha) x (128 + 32 + 2K
// + 2) of its base, inside int16 for sigma_max + alpha <= kKzMaxStep.
//
// Work between window events.  Opens and closes of the 64 lane-halves are the
// only points where a lane-half's state changes kind; between them every
// iteration runs the same row step.  The warp finds its next event with one
// reduce-min and runs the rows up to it without checks.
#pragma once

#include "ga_banded.cuh"
#include "ga_longpk.cuh"

namespace ga {

constexpr int kKzDmin = 128;            // the FIFO's lag bound (>= 127)
// Largest sigma_max + alpha of the packed band kernel (larger scorings run
// kc_kernel in int32): (sigma_max + alpha) x (128 + 32 + 2K + 2) stays far
// inside int16 with room for -inf.
constexpr int kKzMaxStep = 24;
constexpr int kKzRenorm = 128;          // iterations between base moves
constexpr int kKzNegAbs = -(1 << 29);   // absolute -inf in the edge FIFO
constexpr int kKzNever = 1 << 30;       // event iteration of a block that does not exist
// Largest max(m + 1, 128) x super-stages + m of a pair: its iterations
// number less than that plus 64, so they stay below kKzNever.
constexpr int kKzMaxSpan = (1 << 30) - 4096;

// One row of a super-stage's right edge as lane 31 produced it: its raw
// packed H and F words (the high halves are the edge) and its high half's
// base; the reader converts to absolute values.
struct KZEdge {
  uint32_t h, f;
  int32_t base, pad;
};

template <int K>
__global__ void __launch_bounds__(128, 3) kz_kernel(const __grid_constant__ KCParams p) {
  constexpr int kWarps = 4;
  constexpr int W = 32 * K;  // columns per half
  constexpr int W2 = 2 * W;  // columns per super-stage
  constexpr int kRing = 256; // row table words per super-stage slot
  constexpr int kFifo = 128; // edge FIFO slots (iterations)

  __shared__ uint32_t row_s[kWarps][3][kRing + 32];  // + a copy of slots 0..31
  __shared__ uint4 selb_s[kWarps][3][W2 / 16];  // one selector byte per column
  __shared__ int2 fabs_s[kWarps][kFifo];        // absolute edge values by iteration
  __shared__ uint32_t frel_s[kWarps][kFifo + 32];  // the same relative to lane 0's base, + a copy of slots 0..31
  __shared__ int2 blk_s[kWarps][2][32];         // per lane-half: first column, first window row
  __shared__ unsigned long long cells_s[kWarps][32];  // region cells entered, per lane

  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int left_lane = (t + 31) & 31, right_lane = (t + 1) & 31;
  uint32_t(*rowr)[kRing + 32] = row_s[warp];
  uint4(*selb)[W2 / 16] = selb_s[warp];
  int2 *fabs = fabs_s[warp];
  uint32_t *frel = frel_s[warp];
  int2 *blk0 = &blk_s[warp][0][t];
  int2 *blk1 = &blk_s[warp][1][t];
  KZEdge *bnd = reinterpret_cast<KZEdge *>(p.bnd) + (size_t)(blockIdx.x * kWarps + warp) * (size_t)p.bnd_stride;
  const int alpha = p.alpha, beta = p.beta;
  const uint32_t NB = pk16(-beta, -beta);
  const uint32_t NAc = pk16(-alpha, -alpha);
  const uint32_t NEGV = pk16(kNeg16, kNeg16);
  const unsigned FULL = 0xffffffffu;
  const int npairs = p.range[1] - p.range[0];
  const bool bisect = p.bis_lo != nullptr;

  for (;;) {
    int task = 0;
    if (t == 0) task = atomicAdd(p.task_counter, 1);
    task = __shfl_sync(FULL, task, 0);
    if (task >= npairs) break;
    const int pid = p.order[p.range[0] + task];
    const int64_t qs = p.q_off[pid], ts = p.t_off[pid];
    const int m = (int)(p.q_off[pid + 1] - qs), n = (int)(p.t_off[pid + 1] - ts);
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
      if (t == 0) {
        if (bisect) {
          p.bis_lo[pid] = p.bis_hi[pid] = 0;
        } else {
          const int len = m + n;
          p.scores[pid] = len ? -(alpha + beta * (len - 1)) : 0;
          if (p.w_used) p.w_used[pid] = w;
        }
      }
      continue;
    }
    const int dn = n - m;
    const int nb = (n + K - 1) / K;      // blocks
    const int nst = (n + W2 - 1) / W2;   // super-stages
    unsigned tries = 0;
    unsigned long long *cells = &cells_s[warp][t];
    *cells = 0ull;

    for (;;) {  // one attempt at band width w
      const int lo = (dn < 0 ? dn : 0) - w;
      const int hi = (dn > 0 ? dn : 0) + w;
      // spacing: a lane-half's left neighbour opens its next window only
      // after the lane-half's last row (window lengths are at most
      // min(m, B)), and the FIFO's lag D - 63 covers a batch loaded ahead
      const int B = hi - lo + K;
      const int D = ::max(kKzDmin, ::min(m, B - 63 * K) + 1);
      auto Ts = [&](int s) -> int { return D * s - 1; };
      // rows any lane-half of super-stage s runs: [rlo(s), rhi(s)]
      auto rlo = [&](int s) -> int { return ::max(1, W2 * s + 1 - hi); };
      auto rhi = [&](int s) -> int {
        const int cbl = ::min(W2 * s + W2 - K, K * (nb - 1));
        return ::min(m, cbl + K - lo);
      };
      // last iteration of lane-half 0's window in super-stage s
      auto z0 = [&](int s) -> int { return Ts(s) + ::min(m, W2 * s + K - lo); };
      // owner of column n: the last block, whose window ends at row m
      const int bown = nb - 1;
      const int s_own = bown / 64, l_own = bown % 64;
      const int nit = Ts(s_own) + m + l_own + 1;
      int S = kNeg32;

      // ---- per lane-half state (h = 0: low halves, h = 1: high halves) ---
      int sh[2], A[2], Z[2];
      bool act[2] = {false, false};
      int base[2] = {0, 0};
      uint32_t sel[K], H[K], E[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        sel[j] = 0u;
        H[j] = NEGV;
        E[j] = NEGV;
      }
      uint32_t Hdiag = NEGV, Hleft = NEGV, Fin = NEGV;
      uint32_t dr = 0u;      // conversion of what this lane sends, to the receiver's base
      int sf = 0;            // lowest super-stage whose rows may still be filled
      int sfifo = 0;         // lane-half 0's super-stage at the next FIFO load
      int sel_filled = -1;   // highest super-stage with a filled selector slot

      // selector bytes of super-stage s (slot s % 3): byte of column c is
      // (code | (code + 8) << 4), sign replication of byte 0 for padding
      auto fill_sel = [&](int s) {
        // lane t builds the bytes of columns W2 s + 32 t .. + 31 from the (at
        // most three) packed words holding them
        const int c0 = W2 * s + 32 * t;
        uint32_t outw[8];
        if (c0 < n) {
          const int64_t pos = ts + c0, last = (ts + n - 1) >> 4;
          const int64_t wi = pos >> 4;
          const uint32_t sh2 = 2u * (uint32_t)(pos & 15);
          const uint32_t w0 = __ldg(p.packed_t + wi);
          const uint32_t w1 = (wi + 1 <= last) ? __ldg(p.packed_t + wi + 1) : 0u;
          const uint32_t w2 = (wi + 2 <= last) ? __ldg(p.packed_t + wi + 2) : 0u;
          const uint32_t cw[2] = {__funnelshift_r(w0, w1, sh2), __funnelshift_r(w1, w2, sh2)};
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            uint32_t o = 0u;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int cc = 4 * k + c;
              const uint32_t code = (cw[cc >> 4] >> (2 * (cc & 15))) & 3u;
              const uint32_t byte = (c0 + cc < n) ? (code | ((code + 8u) << 4)) : 0x88u;
              o |= byte << (8 * c);
            }
            outw[k] = o;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) outw[k] = 0x88888888u;
        }
        selb[s % 3][2 * t] = make_uint4(outw[0], outw[1], outw[2], outw[3]);
        selb[s % 3][2 * t + 1] = make_uint4(outw[4], outw[5], outw[6], outw[7]);
      };
      // table words of the rows lane-half 0 of super-stage s runs at
      // iterations X .. X + 31
      auto fill_rows = [&](int s, int X) {
        const int r = X + t - Ts(s);
        uint32_t v = 0u;
        if (r >= 1 && r <= m) v = p.tables[packed_code(p.packed_q, qs + r - 1)];
        const int x = r & (kRing - 1);
        rowr[s % 3][x] = v;
        if (x < 32) rowr[s % 3][x + kRing] = v;  // a segment reads up to 32 slots on
      };
      auto fill_rows_for = [&](int X) {
        while (sf < nst && X > Ts(sf) + rhi(sf)) ++sf;
        for (int s = sf; s < nst && Ts(s) + rlo(s) <= X + 31; ++s) fill_rows(s, X);
      };
      auto rel_pack = [&](int2 v, int b) -> uint32_t {
        const int hv = (v.x <= kKzNegAbs) ? kNeg16 : ::min(::max(v.x - b, kNeg16), 32767);
        const int fv = (v.y <= kKzNegAbs) ? kNeg16 : ::min(::max(v.y - b, kNeg16), 32767);
        return pk16(hv, fv);
      };
      auto put_frel = [&](int x, uint32_t v) {
        frel[x] = v;
        if (x < 32) frel[x + kFifo] = v;  // a segment reads up to 32 slots on
      };
      // the left input of lane-half 0 at iterations Y .. Y + 31: the previous
      // super-stage's right edge (or column 0), -inf outside the left
      // block's window
      auto load_fifo = [&](int Y) {
        while (sfifo < nst && Y > z0(sfifo)) ++sfifo;
        const int itf = Y + t;
        int s = sfifo;
        if (s < nst && itf > z0(s)) ++s;
        int2 v = make_int2(kKzNegAbs, kKzNegAbs);
        if (s < nst) {
          const int r = itf - Ts(s);
          if (s == 0) {
            if (r >= 1 && r <= ::min(m, -lo)) {
              const int hv = -alpha - beta * (r - 1);
              v = make_int2(hv, hv - alpha);
            }
          } else {
            const int cbp = W2 * s - K;
            const int plo = ::max(1, cbp + 1 - hi), phi = ::min(m, cbp + K - lo);
            if (r >= plo && r <= phi) {
              const KZEdge e = bnd[r];
              v = make_int2(hi16(e.h) + e.base, hi16(e.f) + e.base);
            }
          }
        }
        fabs[itf & (kFifo - 1)] = v;
        const int b0l = __shfl_sync(FULL, base[0], 0);
        put_frel(itf & (kFifo - 1), rel_pack(v, b0l));
      };
      // lane-half h waits for its window of super-stage s
      auto enter = [&](int h, int s) {
        const int l = t + 32 * h;
        sh[h] = s;
        const int cb = W2 * s + W * h + K * t;
        if (s < nst && cb < n) {
          const int wlo = ::max(1, cb + 1 - hi), whi = ::min(m, cb + K - lo);
          A[h] = Ts(s) + wlo + l;
          Z[h] = Ts(s) + whi + l;
          *(h ? blk1 : blk0) = make_int2(cb, wlo);
          *cells += (unsigned long long)(whi - wlo + 1) * (unsigned long long)::min(K, n - cb);
          uint4 v = selb[s % 3][32 * h + t];
          if (h) {
            v.x += 0x44444444u;
            v.y += 0x44444444u;
            v.z += 0x44444444u;
            v.w += 0x44444444u;
          }
          const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const uint32_t b = (uint32_t)(4 + (j & 3));
            const uint32_t code = h ? (0u | (b << 4) | (2u << 8) | (3u << 12)) : (b | (1u << 4) | (2u << 8) | (3u << 12));
            sel[j] = prmt(sel[j], vw[(j >> 2) & 3], code);
          }
        } else {
          A[h] = kKzNever;
          Z[h] = kKzNever;
          *(h ? blk1 : blk0) = make_int2(0, 1);
        }
      };
      auto row0_h = [&](int c) -> int { return -alpha - beta * (c - 1); };  // H(0, c), c >= 1
      // the receiver's base and activity decide what this lane sends
      auto recompute_dr = [&]() {
        const int rb0 = __shfl_sync(FULL, base[0], right_lane);
        const int rb1 = __shfl_sync(FULL, base[1], right_lane);
        const int ra = __shfl_sync(FULL, (act[0] ? 1 : 0) | (act[1] ? 2 : 0), right_lane);
        int d0 = 0, d1 = 0;
        if (t < 31) {
          if (act[0] && (ra & 1)) d0 = base[0] - rb0;
          if (act[1] && (ra & 2)) d1 = base[1] - rb1;
        } else if (act[0] && (ra & 2)) {  // lane 31's low half feeds lane 0's high half
          d0 = base[0] - rb1;
        }
        dr = pk16(d0, d1);
      };

      // ---- set-up: selectors of super-stages 0 and 1, rows and FIFO of the
      // first iterations, every lane-half waiting for super-stage 0 --------
      __syncwarp();
      fill_sel(0);
      if (nst > 1) fill_sel(1);
      sel_filled = nst > 1 ? 1 : 0;
      __syncwarp();
      enter(0, 0);
      enter(1, 0);
      fill_rows_for(0);
      fill_rows_for(32);
      load_fifo(0);
      __syncwarp();

      int it = 0;
      while (it < nit) {
        if ((it & 31) == 0) {
          __syncwarp();
          if ((it & (kKzRenorm - 1)) == 0 && it > 0) {
            // every lane-half inside its window moves its base to its H of
            // the first column; held values follow their own base (inside)
            // or the left neighbour's (idle: values received unconverted)
            int d0 = 0, d1 = 0;
            if (act[0]) {
              const int v = lo16(H[0]);
              if (v > kNeg16 + 4096) d0 = v;
            }
            if (act[1]) {
              const int v = hi16(H[0]);
              if (v > kNeg16 + 4096) d1 = v;
            }
            base[0] += d0;
            base[1] += d1;
            const uint32_t dm = pk16(d0, d1);
            const uint32_t dlf = __shfl_sync(FULL, dm, left_lane);
            // lane 0's low half holds FIFO values relative to its own base;
            // lane 0's high half receives from lane 31's low half
            const int l0 = (t == 0 || act[0]) ? d0 : lo16(dlf);
            const int l1 = act[1] ? d1 : (t == 0 ? lo16(dlf) : hi16(dlf));
            const uint32_t dh = pk16(l0, l1);
#pragma unroll
            for (int j = 0; j < K; ++j) {
              H[j] = __vmaxs2(__vsubss2(H[j], dm), NEGV);
              E[j] = __vmaxs2(__vsubss2(E[j], dm), NEGV);
            }
            Hdiag = __vmaxs2(__vsubss2(Hdiag, dh), NEGV);
            Hleft = __vmaxs2(__vsubss2(Hleft, dh), NEGV);
            Fin = __vmaxs2(__vsubss2(Fin, dh), NEGV);
            // FIFO entries of this batch, relative to lane 0's new base
            const int b0l = __shfl_sync(FULL, base[0], 0);
            put_frel((it + t) & (kFifo - 1), rel_pack(fabs[(it + t) & (kFifo - 1)], b0l));
            recompute_dr();
          }
          fill_rows_for(it + 64);
          {
            const int s0 = __shfl_sync(FULL, sh[0], 0);  // lane-half 0's super-stage
            while (sel_filled + 1 < nst && sel_filled < s0 + 1) fill_sel(++sel_filled);
          }
          load_fifo(it + 32);
          __syncwarp();
        }
        // ---- window events at the start of iteration it ------------------
        const bool c0 = act[0] && it == Z[0] + 1, c1 = act[1] && it == Z[1] + 1;
        if (__any_sync(FULL, c0 || c1 || (!act[0] && it == A[0]) || (!act[1] && it == A[1]))) {
          // closes first: a lane-half's next window may open at the same
          // iteration
          if (c0) {
            act[0] = false;
            enter(0, sh[0] + 1);
          }
          if (c1) {
            act[1] = false;
            enter(1, sh[1] + 1);
          }
          const bool o0 = !act[0] && it == A[0], o1 = !act[1] && it == A[1];
          const int lb0 = __shfl_sync(FULL, base[0], left_lane);
          const int lb1 = __shfl_sync(FULL, base[1], left_lane);
          if (o0 || o1) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (!(h ? o1 : o0)) continue;
              const uint32_t keep = h ? 0x0000ffffu : 0xffff0000u;
              const int2 bk = *(h ? blk1 : blk0);
              const int cb = bk.x, wlo = bk.y;
              int bn;
              if (t == 0 && h == 0) {
                const int2 e = fabs[it & (kFifo - 1)];
                const int2 e1 = (it > 0) ? fabs[(it - 1) & (kFifo - 1)] : make_int2(kKzNegAbs, kKzNegAbs);
                bn = (e.x > kKzNegAbs) ? e.x : (e1.x > kKzNegAbs ? e1.x : (wlo == 1 ? row0_h(cb + 1) : base[0]));
              } else {
                bn = (t == 0) ? lb0 : (h ? lb1 : lb0);
              }
              base[h] = bn;
              act[h] = true;
#pragma unroll
              for (int j = 0; j < K; ++j) {
                int hv = kNeg16, ev = kNeg16;
                if (wlo == 1) {  // row 0 of the block
                  hv = row0_h(cb + j + 1) - bn;
                  ev = hv - alpha;
                }
                H[j] = (H[j] & keep) | (pk16(hv, hv) & ~keep);
                E[j] = (E[j] & keep) | (pk16(ev, ev) & ~keep);
              }
              const int plo = (cb == 0) ? 0 : ::max(1, cb - K + 1 - hi);
              if (t == 0 && h == 0) {
                // the left input of rows wlo - 1 and wlo from the edge FIFO
                const uint32_t wcur = rel_pack(fabs[it & (kFifo - 1)], bn);
                const uint32_t wprv = rel_pack(fabs[(it - 1) & (kFifo - 1)], bn);
                int hd = lo16(wprv);
                if (wlo - 1 == 0) hd = (cb == 0) ? -bn : ((plo == 1) ? row0_h(cb) - bn : kNeg16);
                Hdiag = (Hdiag & keep) | (pk16(hd, hd) & ~keep);
                Hleft = (Hleft & keep) | (pk16(lo16(wcur), 0) & ~keep);
                Fin = (Fin & keep) | (pk16(hi16(wcur), 0) & ~keep);
              } else if (wlo - 1 == 0) {
                const int hd = (plo == 1) ? row0_h(cb) - bn : kNeg16;
                Hdiag = (Hdiag & keep) | (pk16(hd, hd) & ~keep);
              }
            }
          }
          // lane 0's FIFO entries relative to its (possibly new) base
          {
            const int b0l = __shfl_sync(FULL, base[0], 0);
            const int s0 = __shfl_sync(FULL, o0 ? 1 : 0, 0);
            if (s0) {
              put_frel(t, rel_pack(fabs[t], b0l));
              put_frel(t + 32, rel_pack(fabs[t + 32], b0l));
              put_frel(t + 64, rel_pack(fabs[t + 64], b0l));
              put_frel(t + 96, rel_pack(fabs[t + 96], b0l));
            }
          }
          recompute_dr();
          __syncwarp();
        }
        // ---- rows up to the warp's next event or batch end -----------------
        int ne = ::min(act[0] ? Z[0] + 1 : A[0], act[1] ? Z[1] + 1 : A[1]);
        ne = (int)__reduce_min_sync(FULL, (unsigned)ne);
        // (at least one row: the loop advances whatever the events say)
        const int seg_end = ::max(::min(::min(ne, (it & ~31) + 32), nit), it + 1);
        const uint32_t actm = (act[0] ? 0x0000ffffu : 0u) | (act[1] ? 0xffff0000u : 0u);
        const bool edge_on = (t == 31) && act[1];
        // a segment stays inside one batch of 32 iterations, so its ring and
        // FIFO entries are contiguous (the rings end in a copy of their
        // first 32 slots)
        const int ro0 = -t - Ts(sh[0]), ro1 = -t - 32 - Ts(sh[1]), b1 = base[1];
        const uint32_t *q0 = rowr[sh[0] % 3] + ((it + ro0) & (kRing - 1));
        const uint32_t *q1 = rowr[sh[1] % 3] + ((it + ro1) & (kRing - 1));
        const uint32_t *fq = frel + ((it + 1) & (kFifo - 1));
        KZEdge *bp = bnd + (edge_on ? it + ro1 : 0);
        for (; it < seg_end; ++it, ++q0, ++q1, ++fq, ++bp) {
          const uint32_t twl = *q0;
          const uint32_t twh = *q1;
          uint32_t unused_best = 0u;
          const uint32_t Fout = pk_row<kModeGlobal, K>(
              H, E, Hdiag, Fin, NB, 0u, unused_best, [&](int j) -> uint32_t { return prmt(twl, twh, sel[j]); },
              [&](int) -> uint32_t { return NAc; });
          const uint32_t Hout = H[K - 1];
          if (edge_on) {
            KZEdge e;
            e.h = Hout;
            e.f = Fout;
            e.base = b1;
            e.pad = 0;
            *bp = e;
          }
          const uint32_t hsnd = (__vadd2(Hout, dr) & actm) | (NEGV & ~actm);
          const uint32_t fsnd = (__vadd2(Fout, dr) & actm) | (NEGV & ~actm);
          uint32_t hs = __shfl_sync(FULL, hsnd, left_lane);
          uint32_t fs = __shfl_sync(FULL, fsnd, left_lane);
          if (t == 0) {
            const uint32_t wv = *fq;
            hs = prmt(wv, hs, 0x5410u);
            fs = prmt(wv, fs, 0x5432u);
          }
          Hdiag = Hleft;
          Hleft = hs;
          Fin = fs;
        }
      }
      __syncwarp();
      // ---- the score: H(m, n) from the owner's state after the last row ---
      {
        const int h_own = (l_own >= 32) ? 1 : 0, t_own = l_own - 32 * h_own;
        const int oj = (n - 1) % K;
        if (t == t_own) {
          uint32_t v = H[0];
#pragma unroll
          for (int j = 1; j < K; ++j)
            if (j == oj) v = H[j];
          S = h_own ? hi16(v) + base[1] : lo16(v) + base[0];
        }
        S = __shfl_sync(FULL, S, t_own);
      }
      // ---- certificate (as kc_kernel) -----------------------------------
      const bool covers = (lo <= -m) && (hi >= n);
      int64_t ub = INT64_MIN;
      if (lo - 1 >= -m) ub = ::max(ub, band_ub(m, n, p.sigma_max_pos, alpha, beta, lo - 1));
      if (hi + 1 <= n) ub = ::max(ub, band_ub(m, n, p.sigma_max_pos, alpha, beta, hi + 1));
      const bool ok = covers || (int64_t)S >= ub;
      if (bisect) {
        if (t == 0) {
          if (ok) p.bis_hi[pid] = w;
          else p.bis_lo[pid] = w + 1;
        }
        break;
      }
      if (ok) {
        if (t == 0) {
          p.scores[pid] = S;
          if (p.w_used) p.w_used[pid] = w;
        }
        break;
      }
      w = (w == 0) ? 1 : 2 * w;
      ++tries;
      __syncwarp();
    }
    unsigned long long c64 = *cells;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c64 += __shfl_xor_sync(FULL, c64, o);
    if (t == 0 && tries) atomicAdd(p.retries, (unsigned long long)tries);
    if (t == 0) atomicAdd(p.cells, c64);
  }
}

}  // namespace ga
