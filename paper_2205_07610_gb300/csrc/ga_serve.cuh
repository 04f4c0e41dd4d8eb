// ga_serve.cuh -- strip-task kernel: one warp computes one strip of 512
// columns of one pair; the strips of a pair run on different warps (and
// SMs) at the same time, each a few dozen rows behind its left neighbour.
//
// This is the paper's multi-stage partitioning of a long alignment (Sec. 3.1:
// submatrices of the target computed left to right) spread over warps
// instead of run by one thread group in sequence: the right edge of strip s
// (H and the outgoing F of its last column, per row) is written to global
// memory in batches of 32 rows and published through a per-strip progress
// counter (release); strip s+1 waits (acquire, bounded) until the rows it
// is about to read are published.  Rows are the shorter sequence, columns
// the longer one.
//
// Tasks come from two device-resident rings: strip 0 of each request from
// the producer's ring (host or init kernel), strip s+1 from a continuation
// ring that the warp running strip s fills once it has published the first
// kSvContRows edge rows, so the next strip rarely waits.  A warp claims a
// task with a compare-and-swap of the ring head only when an entry is
// there, continuations first, so a claim is always made by a running warp,
// and the producer of every edge a warp waits on (strip s of the same
// request) was claimed earlier by a warp that is running: the waits end
// without any assumption about which blocks are resident.  Every wait is
// bounded (globaltimer): an edge wait that runs out marks the request
// GA_ERR_TIMEOUT and continues; a warp without work exits once no request
// is in flight and `stop` is set or it has idled for idle_ns, and in any
// case after wait_ns without a claimable task.
//
// A request completes when its last strip finishes: that warp writes the
// score to `out` (if set) and a completion record (id, score, status, seq)
// to the completion ring, seq last.
//
// Substitution scores come from a per-warp int8 profile of the strip in
// shared memory, P[c][x] = sigma(row residue c, column x), for any alphabet
// of <= 31 symbols (Sec. 3.1, "scoring profile").
//
// Cells.  A request whose scoring has sigma_max + alpha <= kSvPkMaxStep runs
// its strips packed (sv_strip_pk): the two 256-column halves of a strip sit
// in the low and high int16 halves of every register, the high half 32 rows
// behind the low one, each value stored relative to a per-lane, per-half
// int32 base that is renormalised every kKwRenorm rows, exactly as in the
// packed long-pair kernel (ga_longpk.cuh: one rotating shuffle, lane 0
// joining the strip's left edge and lane 31's low half, virtual rows before
// the high half's first row, local mode's zero folded into E).  Other
// scorings run the int32 strip (sv_strip).  Strip edges are absolute int32
// in both, so the two strip kinds share the edge and progress protocol.
#pragma once

#include "ga_dp.cuh"
#include "ga_longpk.cuh"

namespace ga {

constexpr int kSvK = 16;
constexpr int kSvKp = 8;          // packed strips: 8 packed columns per lane and half
constexpr int kSvPkMaxStep = 128; // largest sigma_max + alpha of a packed strip
constexpr int kSvW = 32 * kSvK;  // columns per strip
constexpr int kSvWarps = 4;      // warps per block
constexpr int kSvMaxStrips = 128;
constexpr int kSvMaxLen = kSvMaxStrips * kSvW;  // longer sequence <= 65536
constexpr int kSvContRows = 96;  // edge rows published before the next strip is queued

struct SvScoring {
  int32_t A, alpha, beta;
  int32_t packed;         // 1: strips run sv_strip_pk (sigma_max + alpha <= kSvPkMaxStep)
  int8_t sigma[32 * 32];  // sigma(query code, target code), A x A row-major
};

struct SvRequest {
  const uint8_t *q;     // device codes
  const uint8_t *t;
  int2 *edges;          // (nstrips - 1) edges of R + 1 int2 each
  int32_t *out;         // nullable: the score is also stored here
  int64_t id;
  int32_t m, n;
  int32_t mode, scoring;
  int32_t nstrips;
  int32_t score;        // local / semi: max over strips (starts 0); global: from the last strip
  int32_t strips_done;
  int32_t status;
  int32_t pad[2];
  int32_t progress[kSvMaxStrips];  // rows of each strip's edge published
};

struct SvCompletion {
  int64_t id;
  int32_t score, status;
  int64_t seq;   // index + 1, written last
  int64_t slot;  // request slot (host bookkeeping)
};

struct SvParams {
  SvRequest *req;
  const SvScoring *scorings;
  const int2 *tasks;  // (slot, strip)
  int64_t task_cap;
  unsigned long long *head;
  const unsigned long long *tail;
  SvCompletion *comp;  // nullable
  int64_t comp_cap;
  unsigned long long *comp_count;
  const int32_t *stop;
  // continuation queue: strip s+1 of a request, pushed by the warp running
  // strip s once that strip has published kSvContRows edge rows (at most one
  // unclaimed continuation per request, so cont_cap >= requests in flight)
  int2 *cont;
  unsigned long long *cont_seq;  // entry i holds a task once cont_seq[i % cap] == i + 1
  int64_t cont_cap;
  unsigned long long *cont_head;
  unsigned long long *cont_tail;
  // requests admitted (published by the producer of the task queue) and
  // completed (counted here): warps stay while some request is in flight
  const unsigned long long *admitted;
  unsigned long long *completed;
  int64_t idle_ns;
  int64_t wait_ns;
  int32_t prof_bytes;  // per warp: (max A + 1) * kSvW (real residues, one pad / virtual row)
  int32_t short_chain; // packed local / global strips: the one-op column chain (pk_row_fc), for
                       // launches of one pair, whose strips each have a scheduler to themselves
};

__device__ __forceinline__ uint64_t sv_now() {
  uint64_t v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}
__device__ __forceinline__ int sv_ld_acquire(const int32_t *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long sv_ld_acquire64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void sv_st_release(int32_t *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void sv_st_release64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int sv_ld_sys(const int32_t *p) {
  int v;
  asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait until *flag >= need (acquire): true once it is, false when
// limit_ns of globaltimer time pass first.  The poll backs off from 32 ns to
// 2 us of __nanosleep.
__device__ __forceinline__ bool sv_wait_at_least(const int32_t *flag, int need, uint64_t limit_ns) {
  if (sv_ld_acquire(flag) >= need) return true;
  const uint64_t t0 = sv_now();
  unsigned ns = 32;
  while (sv_ld_acquire(flag) < need) {
    if (sv_now() - t0 > limit_ns) return false;
    __nanosleep(ns);
    if (ns < 2048) ns *= 2;
  }
  return true;
}

struct SvView {
  const uint8_t *rowraw, *colraw;
  int2 *edges;
  int R, C, sw, A, alpha, beta, nstrips, packed;
  const int8_t *sigma;
};

// One strip of one request; returns the strip's contribution to the score
// (local: best H; semi: max of row R; global: H(R, C) on the lane that owns
// column C, else INT_MIN).
template <int MODE>
__device__ int sv_strip(const SvParams &p, SvRequest *rq, int slot, const SvView &v, int s, int t,
                        uint8_t *prof, uint8_t *colc, int2 *in_ring, int2 *out_ring,
                        uint32_t *row_ring) {
  using Cell = CellS32;
  using T = int32_t;
  constexpr int K = kSvK, W = kSvW;
  constexpr int kNeg = kNeg32;
  const int R = v.R, C = v.C, A = v.A, alpha = v.alpha, beta = v.beta;
  const T NB = -beta;
  const int col0 = s * W;
  const int2 *edge_in = (s > 0) ? v.edges + (size_t)(s - 1) * (size_t)(R + 1) : nullptr;
  int2 *edge_out = (s + 1 < v.nstrips) ? v.edges + (size_t)s * (size_t)(R + 1) : nullptr;

  // ---- column codes and the strip's profile ---------------------------
  for (int x = t; x < W; x += 32) {
    const int col = col0 + x;
    int c = A;  // pad
    if (col < C) {
      c = __ldcg(v.colraw + col);
      if (c >= A) {
        atomicCAS(&rq->status, 0, GA_ERR_RESIDUE);
        c = A;
      }
    }
    colc[x] = (uint8_t)c;
  }
  __syncwarp();
  // rows c < A only: pad rows (beyond R) are never computed, pad columns
  // (beyond C) read 0 from their own entries
  for (int e = t; e < A * W; e += 32) {
    const int c = e / W, x = e - c * W;
    const int cc = colc[x];
    int val = 0;
    if (c < A && cc < A) val = v.sw ? v.sigma[cc * A + c] : v.sigma[c * A + cc];
    prof[e] = (uint8_t)(int8_t)val;
  }

  T na[MODE == kModeSemi ? K : 1];
  T H[K], E[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int col = col0 + t * K + j;
    if constexpr (MODE == kModeSemi) na[j] = (col == C - 1) ? 0 : -alpha;
    H[j] = (MODE == kModeGlobal) ? ::max(-alpha - beta * col, kNeg) : 0;  // H(0, col+1)
    E[j] = ::max(H[j] - alpha, kNeg);
  }
  const int ocol = C - 1 - col0 - t * K;  // local index of column C, if in this tile
  T best = 0;
  int rowmax = 0, gscore = INT_MIN;

  auto left_row = [&](int r) -> int2 {  // (H(r, col0), F(r, col0+1))
    int2 lv;
    if (s == 0) {
      lv.x = (MODE == kModeGlobal) ? ((r == 0) ? 0 : ::max(-alpha - beta * (r - 1), kNeg)) : 0;
      lv.y = ::max(lv.x - alpha, kNeg);
    } else {
      lv = in_ring[(r - 1) & 63];
    }
    return lv;
  };
  // rows 32b+1 .. 32b+32 of the left edge -> in_ring, after waiting for them
  auto load_batch = [&](int b) {
    if (s == 0) return;
    const int need = ::min(R, 32 * b + 32);
    if (32 * b + 1 > R) return;
    const int32_t *pp = &rq->progress[s - 1];
    if (t == 0 && !sv_wait_at_least(pp, need, (uint64_t)p.wait_ns)) atomicCAS(&rq->status, 0, GA_ERR_TIMEOUT);
    __syncwarp();
    (void)sv_ld_acquire(pp);  // every lane orders its edge loads after the flag
    const int r = 32 * b + 1 + t;
    if (r <= R) in_ring[(r - 1) & 63] = __ldcg(edge_in + r);
  };
  auto fill_rows = [&](int b) {  // row codes, 4 batches of 32 in flight
    const int r = 32 * b + 1 + t;
    uint32_t c = (uint32_t)A;
    if (r <= R) {
      c = __ldcg(v.rowraw + r - 1);
      if (c >= (uint32_t)A) {  // reported; any in-range row keeps the profile read in bounds
        atomicCAS(&rq->status, 0, GA_ERR_RESIDUE);
        c = 0;
      }
    }
    row_ring[r & 127] = c;
  };
  bool queued = false;  // strip s+1 queued
  auto publish = [&](int rows) {  // edge rows 1..rows are in global memory
    __threadfence();
    __syncwarp();
    if (t == 0) {
      sv_st_release(&rq->progress[s], rows);
      if (!queued && rows >= ::min(R, kSvContRows)) {
        const unsigned long long idx = atomicAdd(p.cont_tail, 1ull);
        const int64_t e = (int64_t)(idx % (unsigned long long)p.cont_cap);
        p.cont[e] = make_int2(slot, s + 1);
        __threadfence();
        sv_st_release64(p.cont_seq + e, idx + 1);
      }
    }
    queued = queued || rows >= ::min(R, kSvContRows);
  };

  load_batch(0);
  fill_rows(0);
  fill_rows(1);
  __syncwarp();

  const int h00 = (MODE == kModeGlobal && col0 > 0) ? ::max(-alpha - beta * (col0 - 1), kNeg) : 0;
  int hdt = 0;  // H(0, col0 + t*K)
  if constexpr (MODE == kModeGlobal)
    hdt = (col0 + t * K == 0) ? 0 : ::max(-alpha - beta * (col0 + t * K - 1), kNeg);
  const int2 l1 = left_row(1);
  T Hdiag = (t == 0) ? h00 : hdt;
  T Hleft = (t == 0) ? l1.x : hdt;
  T Fin = (t == 0) ? l1.y : kNeg;

  const int nit = R + 31;
  int flushed = 0;  // edge rows 1..flushed are in global memory
  for (int it = 0; it < nit; ++it) {
    if ((it & 31) == 0) {
      __syncwarp();
      load_batch(it / 32 + 1);
      fill_rows(it / 32 + 2);
      if (it >= 32 && edge_out) {  // lane 31's rows stored since the last flush: .. it-31
        const int r = flushed + 1 + t;
        if (r <= it - 31) edge_out[r] = out_ring[(r - 1) & 31];
        flushed = it - 31;
        publish(flushed);
      }
      __syncwarp();
    }
    const int r = it - t + 1;
    T Hout, Fout;
    if ((unsigned)(r - 1) < (unsigned)R) {
      const uint32_t rv = row_ring[r & 127];
      const uint4 *pr = reinterpret_cast<const uint4 *>(prof + (size_t)rv * W + t * K);
      const uint4 q4 = *pr;
      const uint32_t w[4] = {q4.x, q4.y, q4.z, q4.w};
      Fout = dp_row<Cell, MODE, K>(
          H, E, Hdiag, Fin, NB, best,
          [&](int j) -> T { return (T)prmt(w[j >> 2], 0u, sext_sel<Cell>(j & 3)); },
          [&](int j) -> T {
            if constexpr (MODE == kModeSemi) return na[j];
            else return -alpha;
          });
      Hout = H[K - 1];
      if (r == R) {
        if constexpr (MODE == kModeGlobal) {
          if (ocol >= 0 && ocol < K) {
            T g = H[0];
#pragma unroll
            for (int j = 1; j < K; ++j)
              if (j == ocol) g = H[j];
            gscore = g;
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
    if (t == 31 && r >= 1 && r <= R) out_ring[(r - 1) & 31] = make_int2(Hout, Fout);
    Hdiag = Hleft;
    Hleft = __shfl_up_sync(0xffffffffu, Hout, 1);
    Fin = __shfl_up_sync(0xffffffffu, Fout, 1);
    if (t == 0) {
      const int2 lv = (it + 2 <= R) ? left_row(it + 2) : make_int2(0, kNeg);
      Hleft = lv.x;
      Fin = lv.y;
    }
  }
  __syncwarp();
  if (edge_out) {  // remaining lane-31 rows, then the whole edge is published
    const int r = flushed + 1 + t;
    if (r <= R) edge_out[r] = out_ring[(r - 1) & 31];
    publish(R);
  }
  __syncwarp();
  if constexpr (MODE == kModeLocal) return group_max<32>(best);
  else if constexpr (MODE == kModeSemi) return group_max<32>(rowmax);
  else return __reduce_max_sync(0xffffffffu, gscore);
}

// One strip of one request in packed int16x2 cells (see the file comment):
// returns what sv_strip returns.
template <int MODE, bool FC>
__device__ int sv_strip_pk(const SvParams &p, SvRequest *rq, int slot, const SvView &v, int s, int t,
                           uint8_t *prof, uint8_t *colc, int2 *in_ring, int2 *out_ring,
                           uint32_t *row_ring /* [128 + 32] */) {
  constexpr int K = kSvKp, WH = 32 * kSvKp, W = kSvW;
  static_assert(2 * WH == W, "a packed strip is two halves of the strip");
  constexpr int kRing = 128;
  const int R = v.R, C = v.C, A = v.A, alpha = v.alpha, beta = v.beta;
  const int col0 = s * W;
  const int2 *edge_in = (s > 0) ? v.edges + (size_t)(s - 1) * (size_t)(R + 1) : nullptr;
  int2 *edge_out = (s + 1 < v.nstrips) ? v.edges + (size_t)s * (size_t)(R + 1) : nullptr;
  const uint32_t NB = pk16(-beta, -beta);
  const uint32_t NAc = pk16(-alpha, -alpha);
  const uint32_t NEGV = pk16(kNeg16, kNeg16);
  auto h0 = [&](int c) -> int { return (MODE == kModeGlobal && c > 0) ? -alpha - beta * (c - 1) : 0; };

  // ---- column codes and the strip's profile: rows 0..A-1 and row A, read
  // by the rows before row 1 and past row R (sigma = -beta in global mode,
  // which leaves row 0 unchanged, else 0; what the rows past R compute is
  // never read in global and semi-global mode) ----------------------------
  for (int x = t; x < W; x += 32) {
    const int col = col0 + x;
    int c = A;  // pad
    if (col < C) {
      c = __ldcg(v.colraw + col);
      if (c >= A) {
        atomicCAS(&rq->status, 0, GA_ERR_RESIDUE);
        c = A;
      }
    }
    colc[x] = (uint8_t)c;
  }
  __syncwarp();
  for (int e = t; e < (A + 1) * W; e += 32) {
    const int c = e / W, x = e - c * W;
    const int cc = colc[x];
    int val = 0;
    if (c < A && cc < A) val = v.sw ? v.sigma[cc * A + c] : v.sigma[c * A + cc];
    else if (c == A && MODE == kModeGlobal) val = -beta;
    prof[e] = (uint8_t)(int8_t)val;
  }

  int b[2];
  b[0] = h0(col0 + t * K + 1);
  b[1] = h0(col0 + WH + t * K + 1);
  uint32_t na[MODE == kModeSemi ? K : 1];
  uint32_t H[K], E[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if constexpr (MODE == kModeSemi) {
      const int c0 = col0 + t * K + j, c1 = c0 + WH;
      na[j] = pk16(c0 == C - 1 ? 0 : -alpha, c1 == C - 1 ? 0 : -alpha);
    }
    const int hv = (MODE == kModeGlobal) ? -beta * j : 0;
    H[j] = pk16(hv, hv);
    const int ev = (MODE == kModeLocal) ? 0 : hv - alpha;
    E[j] = pk16(ev, ev);
  }
  uint32_t Z = 0;
  uint32_t D = pk16(t == 0 ? 0 : h0(col0 + t * K + 1 - K) - b[0], h0(col0 + WH + t * K + 1 - K) - b[1]);
  const int ocol = C - 1 - col0;
  const int ohalf = ocol >= WH ? 1 : 0;
  const bool owner = ocol >= 0 && ocol < W && t == (ocol - ohalf * WH) / K;
  const int oj = (ocol - ohalf * WH) % K;
  uint32_t best = 0;
  int best_abs = 0, rowmax = 0, gscore = INT_MIN;

  auto left_row = [&](int r) -> int2 {  // (H(r, col0), F(r, col0 + 1)), absolute
    int2 lv;
    if (s == 0) {
      lv.x = (MODE == kModeGlobal) ? ((r == 0) ? 0 : -alpha - beta * (r - 1)) : 0;
      lv.y = lv.x - alpha;
    } else {
      lv = in_ring[(r - 1) & 63];
    }
    return lv;
  };
  auto load_batch = [&](int bb) {  // left edge rows 32bb+1 .. 32bb+32, after waiting for them
    if (s == 0) return;
    const int need = ::min(R, 32 * bb + 32);
    if (32 * bb + 1 > R) return;
    const int32_t *pp = &rq->progress[s - 1];
    if (t == 0 && !sv_wait_at_least(pp, need, (uint64_t)p.wait_ns)) atomicCAS(&rq->status, 0, GA_ERR_TIMEOUT);
    __syncwarp();
    (void)sv_ld_acquire(pp);
    const int r = 32 * bb + 1 + t;
    if (r <= R) in_ring[(r - 1) & 63] = __ldcg(edge_in + r);
  };
  // row codes (pad code A past the last row) of batch bb, rows 32bb+1 ..
  // 32bb+32: read_rows issues the global load a batch before put_rows
  // stores it, so the load's latency overlaps a batch of rows
  auto read_rows = [&](int bb) -> uint32_t {
    const int r = 32 * bb + 1 + t;
    return (r <= R) ? (uint32_t)__ldcg(v.rowraw + r - 1) : (uint32_t)A;
  };
  // The ring holds each row's profile byte offset (code x W); its first 32
  // entries are mirrored after the last, so that the 32 rows a lane reads in
  // a batch are contiguous.
  auto put_rows = [&](int bb, uint32_t c) {
    const int r = 32 * bb + 1 + t;
    if (c >= (uint32_t)A && r <= R) {
      atomicCAS(&rq->status, 0, GA_ERR_RESIDUE);
      c = 0;
    }
    const int x = r & (kRing - 1);
    row_ring[x] = c * (uint32_t)W;
    if (x < 32) row_ring[x + kRing] = c * (uint32_t)W;
  };
  bool queued = false;
  auto publish = [&](int rows) {
    __threadfence();
    __syncwarp();
    if (t == 0) {
      sv_st_release(&rq->progress[s], rows);
      if (!queued && rows >= ::min(R, kSvContRows)) {
        const unsigned long long idx = atomicAdd(p.cont_tail, 1ull);
        const int64_t e = (int64_t)(idx % (unsigned long long)p.cont_cap);
        p.cont[e] = make_int2(slot, s + 1);
        __threadfence();
        sv_st_release64(p.cont_seq + e, idx + 1);
      }
    }
    queued = queued || rows >= ::min(R, kSvContRows);
  };

  row_ring[(-t) & (kRing - 1)] = (uint32_t)(A * W);  // rows 0 .. -31: virtual
  if (t == 0) row_ring[kRing] = (uint32_t)(A * W);
  load_batch(0);
  put_rows(0, read_rows(0));
  uint32_t next_rows = read_rows(1);  // stored at iteration 0
  __syncwarp();

  const int hd0 = h0(col0 + t * K) - b[0], hd1 = h0(col0 + WH + t * K) - b[1];
  uint32_t Hdiag = pk16(hd0, hd1);
  uint32_t Hleft = Hdiag;
  uint32_t Fin = NEGV;
  if (t == 0) {
    const int2 l1 = left_row(1);
    Hleft = pk16(l1.x - b[0], hd1);
    Fin = pk16(l1.y - b[0], kNeg16);
  }

  // Lane 31's high-half output rows (H and F of the strip's last column) are
  // kept as raw packed words and turned into absolute edge values when they
  // are flushed, with lane 31's high-half base: every batch flushes all rows
  // stored before it, ahead of any renormalisation.
  const bool keep_out = (t == 31) && edge_out != nullptr;
  auto flush_rows = [&](int first, int last_row) {  // at most 32 rows, lane t: row first + t
    const int b31 = __shfl_sync(0xffffffffu, b[1], 31);
    const int r = first + t;
    if (r <= last_row) {
      const int2 o = out_ring[(r - 1) & 31];
      edge_out[r] = make_int2(hi16((uint32_t)o.x) + b31, hi16((uint32_t)o.y) + b31);
    }
  };
  const uint8_t *prof_lo = prof + t * K, *prof_hi = prof + WH + t * K;

  // One row step of this lane.  GENERAL: some lane of the warp is before row
  // 1, past row R or at row R, lane 31's output row or lane 0's next edge
  // row is outside 1..R; the other batches of 32 steps run without checks.
  auto step = [&](int it, uint32_t off_lo, uint32_t off_hi, auto general_tag) {
    constexpr bool GENERAL = decltype(general_tag)::value;
    // lane 0's next left input (the strip's left edge at row it + 2), read
    // before the row update so that it is ready when the shuffles are
    int lx = kNeg16, ly = kNeg16;
    if (t == 0 && (!GENERAL || it + 2 <= R)) {
      const int2 lv = left_row(it + 2);
      lx = lv.x - b[0];
      ly = lv.y - b[0];
    }
    const int rlo = it - t + 1, rhi = rlo - 32;
    uint32_t Hout, Fout;
    if (!GENERAL || rlo >= 1) {
      const uint2 wl = *reinterpret_cast<const uint2 *>(prof_lo + off_lo);
      const uint2 wh = *reinterpret_cast<const uint2 *>(prof_hi + off_hi);
      auto sig = [&](int j) -> uint32_t {
        return prmt(j < 4 ? wl.x : wl.y, j < 4 ? wh.x : wh.y, sext_sel<CellS16x2>(j & 3));
      };
      if constexpr (FC && MODE != kModeSemi)
        Fout = pk_row_fc<MODE, K>(H, E, Hdiag, Fin, NB, NAc, Z, best, sig);
      else
        Fout = pk_row<MODE, K>(H, E, Hdiag, Fin, NB, Z, best, sig, [&](int j) -> uint32_t {
          if constexpr (MODE == kModeSemi) return na[j];
          else return NAc;
        });
      Hout = H[K - 1];
      if constexpr (GENERAL && MODE != kModeLocal) {
        if (rlo == R || rhi == R) {
          const int h = (rhi == R) ? 1 : 0;
          if constexpr (MODE == kModeGlobal) {
            if (owner && h == ohalf) {
              uint32_t g = H[0];
#pragma unroll
              for (int j = 1; j < K; ++j)
                if (j == oj) g = H[j];
              gscore = h ? hi16(g) + b[1] : lo16(g) + b[0];
            }
          } else {
            uint32_t mx = H[0];
#pragma unroll
            for (int j = 1; j < K; ++j) mx = __vmaxs2(mx, H[j]);
            rowmax = ::max(rowmax, h ? hi16(mx) + b[1] : lo16(mx) + b[0]);
          }
        }
      }
    } else {
      Hout = H[K - 1];
      Fout = NEGV;
    }
    if (keep_out && (!GENERAL || (rhi >= 1 && rhi <= R)))
      out_ring[(rhi - 1) & 31] = make_int2((int)Hout, (int)Fout);
    Hdiag = Hleft;
    uint32_t hs = __shfl_sync(0xffffffffu, Hout, (t + 31) & 31);
    uint32_t fs = __shfl_sync(0xffffffffu, Fout, (t + 31) & 31);
    if (t == 0) {
      hs = prmt((uint32_t)lx, hs, 0x5410u);
      fs = prmt((uint32_t)ly, fs, 0x5410u);
    }
    Hleft = __vadd2(hs, D);
    Fin = __vadd2(fs, D);
  };

  const int nit = R + 63;
  int flushed = 0;  // edge rows 1..flushed are in global memory
  for (int it0 = 0; it0 < nit; it0 += 32) {
    __syncwarp();
    load_batch(it0 / 32 + 1);
    put_rows(it0 / 32 + 1, next_rows);
    next_rows = read_rows(it0 / 32 + 2);
    if (it0 >= 64 && edge_out) {  // lane 31's high-half rows stored since the last flush: .. it0-63
      flush_rows(flushed + 1, it0 - 63);
      flushed = it0 - 63;
      publish(flushed);
    }
    if ((it0 & (kKwRenorm - 1)) == 0 && it0 > 0) {
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
      if constexpr (MODE == kModeLocal) {
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
  if (edge_out) {
    flush_rows(flushed + 1, R);
    publish(R);
  }
  __syncwarp();
  if constexpr (MODE == kModeLocal) {
    best_abs = ::max(best_abs, ::max(lo16(best) + b[0], hi16(best) + b[1]));
    return group_max<32>(best_abs);
  } else if constexpr (MODE == kModeSemi) {
    return group_max<32>(rowmax);
  } else {
    return __reduce_max_sync(0xffffffffu, gscore);
  }
}

__global__ void __launch_bounds__(32 * kSvWarps) ks_kernel(const __grid_constant__ SvParams p) {
  extern __shared__ __align__(16) uint8_t sv_smem[];
  // Static shared memory is kept small so that four blocks fit on an SM
  // with a 24-symbol profile: a strip's column codes are needed only while
  // its profile is built, before the left-edge ring is first written, so
  // the two share their bytes.
  __shared__ int2 in_ring_s[kSvWarps][64];
  __shared__ int2 out_ring_s[kSvWarps][32];
  __shared__ uint32_t row_ring_s[kSvWarps][128 + 32];
  static_assert(sizeof(in_ring_s[0]) >= kSvW, "column codes fit in the left-edge ring");
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  uint8_t *prof = sv_smem + (size_t)warp * (size_t)p.prof_bytes;
  uint8_t *colc = reinterpret_cast<uint8_t *>(in_ring_s[warp]);

  for (;;) {
    // ---- claim the next task (lane 0), bounded idle wait ----------------
    int slot = -1, strip = 0, quit = 0;
    if (t == 0) {
      uint64_t idle0 = 0;
      unsigned ns = 64;
      for (;;) {
        // continuations first: they belong to requests already running
        const unsigned long long ch = *(volatile unsigned long long *)p.cont_head;
        if (ch < sv_ld_acquire64(p.cont_tail)) {
          const int64_t e = (int64_t)(ch % (unsigned long long)p.cont_cap);
          if (sv_ld_acquire64(p.cont_seq + e) == ch + 1) {
            if (atomicCAS(p.cont_head, ch, ch + 1) == ch) {
              const int2 tk = __ldcg(p.cont + e);
              slot = tk.x;
              strip = tk.y;
              break;
            }
            continue;
          }
        }
        const unsigned long long tl = sv_ld_acquire64(p.tail);
        const unsigned long long h = *(volatile unsigned long long *)p.head;
        if (h < tl) {
          if (atomicCAS(p.head, h, h + 1) == h) {
            const int2 tk = __ldcg(p.tasks + (int64_t)(h % (unsigned long long)p.task_cap));
            slot = tk.x;
            strip = tk.y;
            break;
          }
          continue;
        }
        // no task: leave once nothing is in flight and the producer has
        // stopped (or has been quiet for idle_ns)
        const bool drained = sv_ld_acquire64(p.admitted) == *(volatile unsigned long long *)p.completed;
        if (drained && sv_ld_sys(p.stop)) {
          quit = 1;
          break;
        }
        const uint64_t now = sv_now();
        if (!idle0) idle0 = now;
        else if (drained && now - idle0 > (uint64_t)p.idle_ns) {
          quit = 1;
          break;
        } else if (now - idle0 > (uint64_t)p.wait_ns) {  // nothing claimable for wait_ns
          quit = 1;
          break;
        }
        __nanosleep(ns);
        if (ns < 4096) ns *= 2;
      }
    }
    quit = __shfl_sync(0xffffffffu, quit, 0);
    if (quit) break;
    slot = __shfl_sync(0xffffffffu, slot, 0);
    strip = __shfl_sync(0xffffffffu, strip, 0);

    SvRequest *rq = p.req + slot;
    const int m = __ldcg(&rq->m), n = __ldcg(&rq->n);
    const int mode = __ldcg(&rq->mode), sc = __ldcg(&rq->scoring);
    SvView v;
    v.sw = m > n;
    v.R = v.sw ? n : m;
    v.C = v.sw ? m : n;
    v.rowraw = v.sw ? (const uint8_t *)__ldcg((const unsigned long long *)&rq->t)
                    : (const uint8_t *)__ldcg((const unsigned long long *)&rq->q);
    v.colraw = v.sw ? (const uint8_t *)__ldcg((const unsigned long long *)&rq->q)
                    : (const uint8_t *)__ldcg((const unsigned long long *)&rq->t);
    v.nstrips = __ldcg(&rq->nstrips);
    v.edges = (int2 *)__ldcg((const unsigned long long *)&rq->edges);
    v.A = __ldcg(&p.scorings[sc].A);
    v.alpha = __ldcg(&p.scorings[sc].alpha);
    v.beta = __ldcg(&p.scorings[sc].beta);
    v.sigma = p.scorings[sc].sigma;
    v.packed = __ldcg(&p.scorings[sc].packed);

    int val;
    if (v.R == 0 || v.C == 0) {  // closed forms, any mode
      const int len = v.R + v.C;
      val = (mode == kModeGlobal && len) ? -(v.alpha + v.beta * (len - 1)) : 0;
    } else if (v.packed) {
      if (mode == kModeLocal && p.short_chain)
        val = sv_strip_pk<kModeLocal, true>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                            out_ring_s[warp], row_ring_s[warp]);
      else if (mode == kModeLocal)
        val = sv_strip_pk<kModeLocal, false>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                             out_ring_s[warp], row_ring_s[warp]);
      else if (mode == kModeGlobal && p.short_chain)
        val = sv_strip_pk<kModeGlobal, true>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                             out_ring_s[warp], row_ring_s[warp]);
      else if (mode == kModeGlobal)
        val = sv_strip_pk<kModeGlobal, false>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                              out_ring_s[warp], row_ring_s[warp]);
      else
        val = sv_strip_pk<kModeSemi, false>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                            out_ring_s[warp], row_ring_s[warp]);
    } else if (mode == kModeLocal) {
      val = sv_strip<kModeLocal>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                 out_ring_s[warp], row_ring_s[warp]);
    } else if (mode == kModeGlobal) {
      val = sv_strip<kModeGlobal>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                  out_ring_s[warp], row_ring_s[warp]);
    } else {
      val = sv_strip<kModeSemi>(p, rq, slot, v, strip, t, prof, colc, in_ring_s[warp],
                                out_ring_s[warp], row_ring_s[warp]);
    }
    if (t == 0) {
      if (mode == kModeGlobal) {
        if (strip + 1 == v.nstrips || v.R == 0 || v.C == 0) atomicExch(&rq->score, val);
      } else {
        atomicMax(&rq->score, val);
      }
      __threadfence();
      const int done = atomicAdd(&rq->strips_done, 1) + 1;
      if (done == v.nstrips) {
        __threadfence();
        atomicAdd(p.completed, 1ull);
        const int score = atomicAdd(&rq->score, 0);
        const int status = atomicAdd(&rq->status, 0);
        int32_t *out = (int32_t *)__ldcg((const unsigned long long *)&rq->out);
        if (out) *out = status ? INT_MIN : score;
        if (p.comp) {
          const unsigned long long idx = atomicAdd(p.comp_count, 1ull);
          SvCompletion *c = p.comp + (int64_t)(idx % (unsigned long long)p.comp_cap);
          c->id = __ldcg(&rq->id);
          c->score = status ? INT_MIN : score;
          c->status = status;
          c->slot = slot;
          __threadfence_system();
          *(volatile int64_t *)&c->seq = (int64_t)idx + 1;
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace ga
